"""The split lattice on the GPU (domain decomposition along t, halo depth 3
for the Naik hops, inner products summed over ranks).

Ranks are emulated in one process by threads that share this one GPU and
exchange through host-side barriers between launches (no kernel waits on
another rank's kernel), and, separately, by two processes on the same GPU
talking through a gloo process group (the torch.distributed communicator,
halos staged through host memory).  The split operator must equal the
oracle's global operator on every rank's own sites, and the split FP64 CG
must reach the oracle's 1e-10 whole-field residual."""

import os
import socket
import threading

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_common import TOL_DSLASH, dev, oracle_true_residual, rel_l2, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


def _stag():
    import paper_1712_00143_gb300 as stag

    return stag


def _thread_comm_class():
    stag = _stag()

    class ThreadComm(stag.Communicator):
        """Ranks as threads of one process: deposit, barrier, copy, barrier."""

        def __init__(self, rank, size, shared):
            super().__init__(rank, size)
            self.sh = shared

        def exchange(self, send_lo, send_hi, recv_lo, recv_hi):
            sh, R, r = self.sh, self.size, self.rank
            sh["lo"][r], sh["hi"][r] = send_lo.clone(), send_hi.clone()
            torch.cuda.current_stream().synchronize()
            sh["barrier"].wait()
            recv_lo.copy_(sh["hi"][(r - 1) % R])
            recv_hi.copy_(sh["lo"][(r + 1) % R])
            torch.cuda.current_stream().synchronize()
            sh["barrier"].wait()

        def allreduce(self, t):
            sh = self.sh
            sh["red"][self.rank] = t.clone()
            torch.cuda.current_stream().synchronize()
            sh["barrier"].wait()
            total = sh["red"][0].clone()
            for k in range(1, self.size):
                total += sh["red"][k]  # the same order on every rank
            t.copy_(total)
            torch.cuda.current_stream().synchronize()
            sh["barrier"].wait()

    return ThreadComm


def _run_ranks(nranks, work):
    """work(rank, comm) in one thread per rank; returns their results."""
    ThreadComm = _thread_comm_class()
    shared = {"lo": [None] * nranks, "hi": [None] * nranks, "red": [None] * nranks,
              "barrier": threading.Barrier(nranks, timeout=120)}
    out, errs = [None] * nranks, []

    def body(r):
        try:
            torch.cuda.set_device(0)
            with torch.cuda.stream(torch.cuda.Stream()):  # each rank its own stream
                out[r] = work(r, ThreadComm(r, nranks, shared))
        except Exception as e:  # noqa: BLE001
            errs.append(e)
            shared["barrier"].abort()

    ts = [threading.Thread(target=body, args=(r,)) for r in range(nranks)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    if errs:
        raise errs[0]
    return out


GDIMS = (4, 6, 4, 16)


@pytest.fixture(scope="module")
def field():
    fat, lng = synth.gauge_field(GDIMS, 0.3, 1060)
    return fat, lng


@pytest.mark.parametrize("nranks", [1, 2, 4])
def test_split_operator_matches_the_oracle(field, nranks):
    stag = _stag()
    fat, lng = field
    psi_e = synth.random_spinor(GDIMS, 71)
    psi_o = synth.random_spinor(GDIMS, 72)
    d_oe = oracle.dslash(fat, lng, psi_e, GDIMS, 1)
    d_eo = oracle.dslash(fat, lng, psi_o, GDIMS, 0)
    m_ref = oracle.apply_m(fat, lng, psi_e, 0.05, GDIMS)

    def work(r, comm):
        fe = dev(stag.dd_slab(fat, GDIMS, r, nranks))
        le = dev(stag.dd_slab(lng, GDIMS, r, nranks))
        h = stag.stag_dd_create(GDIMS, r, nranks, fe, le)
        outs = []
        for parity, src in ((1, psi_e), (0, psi_o)):
            x = dev(stag.dd_own_sites(src, GDIMS, r, nranks))
            y = torch.empty_like(x)
            stag.stag_dd_dslash(h, y, x, parity, comm)
            outs.append(y.cpu().numpy())
        x = dev(stag.dd_own_sites(psi_e, GDIMS, r, nranks))
        y = torch.empty_like(x)
        stag.stag_dd_apply_m(h, y, x, 0.05, comm)
        outs.append(y.cpu().numpy())
        h.free()
        return outs

    res = _run_ranks(nranks, work)
    for k, ref in enumerate((d_oe, d_eo, m_ref)):
        got = np.concatenate([res[r][k] for r in range(nranks)])
        assert rel_l2(got, ref) < TOL_DSLASH["fp64"], (nranks, k)


@pytest.mark.parametrize("nranks", [2, 4])
def test_split_cg_reaches_the_oracle_residual(field, nranks):
    stag = _stag()
    fat, lng = field
    mass = 0.05
    b = synth.gaussian_source(GDIMS, 5600)

    def work(r, comm):
        fe = dev(stag.dd_slab(fat, GDIMS, r, nranks))
        le = dev(stag.dd_slab(lng, GDIMS, r, nranks))
        h = stag.stag_dd_create(GDIMS, r, nranks, fe, le)
        bl = dev(stag.dd_own_sites(b, GDIMS, r, nranks))
        x = torch.zeros_like(bl)
        info = stag.stag_dd_cg(h, x, bl, mass, comm, tol=1e-10)
        h.free()
        return x.cpu().numpy(), info

    res = _run_ranks(nranks, work)
    x = np.concatenate([res[r][0] for r in range(nranks)])
    infos = [res[r][1] for r in range(nranks)]
    assert all(i["converged"] and i["return"] == 0 for i in infos), infos
    assert len({i["iters"] for i in infos}) == 1  # every rank took the same iterations
    resid = oracle_true_residual(fat, lng, x, b, mass, GDIMS)
    print(f"split CG on {nranks} ranks: {infos[0]['iters']} iterations, oracle residual {resid:.2e}")
    assert resid <= 1e-10
    # the single-lattice FP64 CG takes the same iterations (to within the
    # rounding of sums taken in a different order)
    h = stag.stag_load_links(GDIMS, dev(fat), dev(lng))
    xs = torch.zeros((h.Vh, 3), dtype=torch.complex128, device="cuda")
    single = stag.stag_cg(h, xs, dev(b), mass, mode="plain64", tol=1e-10)
    h.free()
    print(f"single-lattice FP64 CG: {single['iters']} iterations")
    assert abs(single["iters"] - infos[0]["iters"]) <= 2, (single["iters"], infos[0]["iters"])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_worker(rank, size, port, outdir):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=size)
    try:
        import paper_1712_00143_gb300 as stag

        torch.cuda.set_device(0)
        fat, lng = synth.gauge_field(GDIMS, 0.3, 1060)
        b = synth.gaussian_source(GDIMS, 5601)
        h = stag.stag_dd_create(GDIMS, rank, size, dev(stag.dd_slab(fat, GDIMS, rank, size)),
                                dev(stag.dd_slab(lng, GDIMS, rank, size)))
        bl = dev(stag.dd_own_sites(b, GDIMS, rank, size))
        x = torch.zeros_like(bl)
        info = stag.stag_dd_cg(h, x, bl, 0.05, stag.TorchDistComm(), tol=1e-10)
        np.save(os.path.join(outdir, f"x{rank}.npy"), x.cpu().numpy())
        np.save(os.path.join(outdir, f"info{rank}.npy"), np.array([info["iters"], info["converged"], info["return"]]))
        h.free()
    finally:
        dist.destroy_process_group()


def test_split_cg_two_processes_gloo(field, tmp_path):
    """Two processes on this one GPU, a gloo process group between them."""
    import torch.multiprocessing as mp

    fat, lng = field
    mp.start_processes(_gloo_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, start_method="spawn")
    x = np.concatenate([np.load(tmp_path / f"x{r}.npy") for r in range(2)])
    infos = [np.load(tmp_path / f"info{r}.npy") for r in range(2)]
    assert all(i[1] == 1 and i[2] == 0 for i in infos) and infos[0][0] == infos[1][0], infos
    b = synth.gaussian_source(GDIMS, 5601)
    resid = oracle_true_residual(fat, lng, x, b, 0.05, GDIMS)
    print(f"split CG, 2 gloo processes: {infos[0][0]} iterations, oracle residual {resid:.2e}")
    assert resid <= 1e-10
