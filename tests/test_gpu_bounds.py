"""The bounds-checked build (libstag_debug.so: every neighbour index of the
stencil, every vector site index and every link site index checked, the
violations recorded in device words) runs the small parity cases on 4^4, 8^4
and the ragged 4x6x8x10: the Dslash in every format with one and several
right-hand sides, the double-float operator, the even-odd operator, a mixed
CG, a batched solve and the split-lattice operator.  It must record no
violation, and its results must still match the oracle.  (compute-sanitizer
is not available to these tests; this build takes its place for the
library's own index arithmetic.)"""

import json
import os
import subprocess
import sys

import pytest

from gpu_common import requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = r'''
import json
import numpy as np
import torch
import oracle
import synth
import paper_1712_00143_gb300 as stag

def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()

def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))

class SelfComm(stag.Communicator):
    def exchange(self, slo, shi, rlo, rhi):
        rlo.copy_(shi)
        rhi.copy_(slo)
    def allreduce(self, t):
        pass

assert stag.stag_bounds_violations(clear=True)[0] == 0
worst = {}
for dims in [(4, 4, 4, 4), (8, 8, 8, 8), (4, 6, 8, 10)]:
    fat, lng = synth.gauge_field(dims, 0.3, 1000)
    for recon in (18, 12):
        h = stag.stag_load_links(dims, dev(fat), dev(lng), recon_long=recon)
        for parity in (0, 1):
            psi = synth.random_spinor(dims, 7 + parity)
            ref = oracle.dslash(fat, lng, psi, dims, parity)
            for prec in ("fp64", "fp32", "fp16", "fx16", "df64", "fx16l"):
                out = torch.empty_like(dev(psi))
                stag.stag_dslash(h, out, dev(psi), parity, prec)
                worst[prec] = max(worst.get(prec, 0.0), rel(out.cpu().numpy(), ref))
        psi = np.stack([synth.random_spinor(dims, 20 + k) for k in range(8)])
        refs = [oracle.dslash(fat, lng, psi[k], dims, 1) for k in range(8)]
        for prec in ("fp32", "fx16", "fx16l", "df64"):
            out = torch.empty(psi.shape, dtype=torch.complex128, device="cuda")
            stag.stag_dslash(h, out, dev(psi), 1, prec, nrhs=8)
            got = out.cpu().numpy()
            worst[prec + "/8"] = max(rel(got[k], refs[k]) for k in range(8))
        v = synth.random_spinor(dims, 31)
        ref = oracle.apply_m(fat, lng, v, 0.1, dims)
        for prec in ("fp64", "df64"):
            out = torch.empty(v.shape, dtype=torch.complex128, device="cuda")
            stag.stag_apply_m(h, out, dev(v), 0.1, prec=prec)
            worst["apply_m/" + prec] = max(worst.get("apply_m/" + prec, 0.0), rel(out.cpu().numpy(), ref))
        b = synth.gaussian_source(dims, 5000)
        x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
        stag.stag_cg(h, x, dev(b), 0.1, mode="mixed32", tol=1e-10)
        worst["cg"] = max(worst.get("cg", 0.0), oracle.true_residual(fat, lng, x.cpu().numpy(), b, 0.1, dims))
        bs = np.stack([synth.gaussian_source(dims, 5100 + k) for k in range(4)])
        xs = torch.zeros(bs.shape, dtype=torch.complex128, device="cuda")
        stag.stag_batch_solve([(h, xs, dev(bs), 4, 0.1)], mode="mixed16l", tol=1e-10)
        xh = xs.cpu().numpy()
        worst["batch"] = max([worst.get("batch", 0.0)] +
                             [oracle.true_residual(fat, lng, xh[k], bs[k], 0.1, dims) for k in range(4)])
        h.free()
    if dims[3] % 2 == 0 and dims[3] >= 4:
        d = stag.stag_dd_create(dims, 0, 1, dev(stag.dd_slab(fat, dims, 0, 1)), dev(stag.dd_slab(lng, dims, 0, 1)))
        v = synth.random_spinor(dims, 41)
        out = torch.empty(v.shape, dtype=torch.complex128, device="cuda")
        stag.stag_dd_apply_m(d, out, dev(v), 0.1, SelfComm(0, 1))
        worst["dd"] = max(worst.get("dd", 0.0), rel(out.cpu().numpy(), oracle.apply_m(fat, lng, v, 0.1, dims)))
        d.free()
n, code, index = stag.stag_bounds_violations()
print(json.dumps({"violations": n, "first_code": code, "first_index": index, "worst": worst}))
'''


def test_bounds_checked_build_records_no_violation():
    sys.path.insert(0, os.path.join(ROOT, "paper_1712_00143_gb300"))
    import build

    lib = build.build(debug_bounds=True)
    env = dict(os.environ, STAG_LIBRARY=lib)
    env["PYTHONPATH"] = os.pathsep.join([ROOT] + [p for p in env.get("PYTHONPATH", "").split(os.pathsep) if p])
    out = subprocess.run([sys.executable, "-c", CASES], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=1800)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-4000:]
    r = json.loads(out.stdout.strip().splitlines()[-1])
    print(r)
    assert r["violations"] == 0, r
    w = r["worst"]
    tol = {"fp64": 1e-13, "df64": 1e-13, "fp32": 1e-6, "fp16": 5e-3, "fx16": 5e-4, "fx16l": 5e-4}
    for k, v in w.items():
        base = k.split("/")[-1] if k.startswith("apply_m") else k.split("/")[0]
        if k in ("cg", "batch"):
            assert v <= 1e-10, (k, v)
        elif k == "dd":
            assert v < 1e-13, (k, v)
        else:
            assert v < tol[base], (k, v)
