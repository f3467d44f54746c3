"""CPU checks of the split-lattice (domain decomposition along t) layout.

(1) The slab convention the library's split operator uses: rank r of R holds
the links of global slices r T - 4 .. r T + T + 3 (periodic) and computes its
own output sites from a field whose halo slices [1, 4) and [T + 4, T + 7) came
from its neighbours; the outermost slice on each side is never read.  The
oracle's Dslash on that extended slab, with the two outermost slices zeroed,
must equal the oracle's global Dslash on the rank's own sites, for R = 1, 2,
3 and both parities.  (2) The torch.distributed communicator's exchange and
sum semantics in world-size 2 and 3 gloo process groups on the CPU."""

import os
import socket

import numpy as np
import pytest
import torch

import oracle
import synth

H = 4


def _stag():
    import paper_1712_00143_gb300 as stag

    return stag


@pytest.mark.parametrize("nranks", [1, 2, 3])
@pytest.mark.parametrize("out_parity", [0, 1])
def test_slab_operator_equals_global_operator(nranks, out_parity):
    stag = _stag()
    gdims = (4, 6, 4, 12)
    fat, lng = synth.gauge_field(gdims, 0.3, 1050)
    psi = synth.random_spinor(gdims, 33)  # lives on parity 1 - out_parity
    ref = oracle.dslash(fat, lng, psi, gdims, out_parity)
    T = gdims[3] // nranks
    S = gdims[0] // 2 * gdims[1] * gdims[2]
    ext = (gdims[0], gdims[1], gdims[2], T + 2 * H)
    for r in range(nranks):
        fe = stag.dd_slab(fat.reshape(-1, 4, 3, 3), gdims, r, nranks)
        le = stag.dd_slab(lng.reshape(-1, 4, 3, 3), gdims, r, nranks)
        # the input field on the extended slab: own sites and the halos an
        # exchange delivers; slices 0 and T + 7 stay zero
        pe = np.zeros((S * (T + 2 * H), 3), dtype=np.complex128)
        for k in range(1, T + 2 * H - 1):
            t = (r * T - H + k) % gdims[3]
            pe[k * S:(k + 1) * S] = psi[t * S:(t + 1) * S]
        own = np.arange(H * S, (H + T) * S)
        got = oracle.dslash(fe.reshape(-1, 4, 3, 3), le.reshape(-1, 4, 3, 3), pe, ext, out_parity, out_sites=own)
        want = stag.dd_own_sites(ref, gdims, r, nranks)
        assert np.abs(got - want).max() < 1e-14 * np.abs(want).max(), (nranks, r)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _comm_worker(rank, size, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=size)
    try:
        import paper_1712_00143_gb300 as stag

        c = stag.TorchDistComm()
        n = 24
        send_lo = torch.full((n,), 10 * rank + 1, dtype=torch.uint8)
        send_hi = torch.full((n,), 10 * rank + 2, dtype=torch.uint8)
        recv_lo = torch.zeros(n, dtype=torch.uint8)
        recv_hi = torch.zeros(n, dtype=torch.uint8)
        c.exchange(send_lo, send_hi, recv_lo, recv_hi)
        vals = torch.tensor([rank + 0.5, 2.0 ** -rank], dtype=torch.float64)
        c.allreduce(vals)
        q.put((rank, int(recv_lo[0]), int(recv_hi[0]), int(recv_lo.min()), int(recv_hi.max()), vals.tolist()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("size", [2, 3])
def test_torch_communicator_exchange_and_sum(size):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    mp.start_processes(_comm_worker, args=(size, _free_port(), q), nprocs=size, start_method="spawn")
    got = sorted(q.get(timeout=60) for _ in range(size))
    want_sum = [sum(r + 0.5 for r in range(size)), sum(2.0 ** -r for r in range(size))]
    for rank, lo0, hi0, lo_min, hi_max, vals in got:
        below, above = (rank - 1) % size, (rank + 1) % size
        assert lo0 == lo_min == 10 * below + 2  # the rank below's send_hi
        assert hi0 == hi_max == 10 * above + 1  # the rank above's send_lo
        assert vals == want_sum
