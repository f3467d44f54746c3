"""Training data and training runs for the learned preconditioner.

Pairs (r_k, e_k) come from the unpreconditioned solver on a gauge field:
for each source b, a reference solution x* (1e-12), then iterates x_k of the
mixed-precision CG stopped after k iterations; r_k = b - M x_k (FP64, on the
GPU) and e_k = x* - x_k.  Everything runs through the library's C ABI.
"""

import torch

from . import stag_apply_m, stag_cg


def make_pairs(h, sources, mass, iters, dtype=torch.complex64, mode="mixed32"):
    """List of (handle, r, e) training pairs; `sources`: complex128 CUDA tensors [V/2][3]."""
    pairs = []
    for b in sources:
        xs = torch.zeros_like(b)
        stag_cg(h, xs, b, mass, mode=mode, tol=1e-12)
        for k in iters:
            xk = torch.zeros_like(b)
            stag_cg(h, xk, b, mass, mode=mode, max_iter=int(k), check_interval=1, raise_on_error=False)
            mx = torch.empty_like(b)
            stag_apply_m(h, mx, xk, mass, prec="fp64")
            r = (b - mx).to(dtype).contiguous()
            e = (xs - xk).to(dtype).contiguous()
            pairs.append((h, r, e))
    return pairs
