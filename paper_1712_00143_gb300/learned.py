"""Training data and training runs for the learned preconditioner.

Pairs (r_k, e_k) come from the unpreconditioned solver on a gauge field:
for each source b, a reference solution x* (1e-12), then a chain of
mixed-precision CG segments from x = 0, each restarted from where the last
one stopped, with a pair taken at the end of every segment (after k
iterations in total): r_k = b - M x_k (FP64, on the GPU) and e_k = x* - x_k.
Everything runs through the library's C ABI.
"""

import torch

from . import stag_apply_m, stag_cg


def make_pairs(h, sources, mass, iters, dtype=torch.complex64, mode="mixed32"):
    """List of (handle, r, e) training pairs; `sources`: complex128 CUDA tensors [V/2][3];
    `iters`: increasing total iteration counts at which pairs are taken."""
    pairs = []
    for b in sources:
        xs = torch.zeros_like(b)
        stag_cg(h, xs, b, mass, mode=mode, tol=1e-12)
        x = torch.zeros_like(b)
        done = 0
        for k in sorted(int(k) for k in iters):
            if k > done:
                stag_cg(h, x, b, mass, mode=mode, max_iter=k - done, check_interval=1, use_initial_guess=1,
                        raise_on_error=False)
                done = k
            mx = torch.empty_like(b)
            stag_apply_m(h, mx, x, mass, prec="fp64")
            r = (b - mx).to(dtype).contiguous()
            e = (xs - x).to(dtype).contiguous()
            pairs.append((h, r, e))
    return pairs
