"""Helpers shared by the GPU parity tests: seeded fixtures on the device."""

import numpy as np
import pytest
import torch

import synth

requires_gpu = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")

# relative L2 error bounds: FP64 1e-13, FP32 1e-6, the 16-bit formats 5e-3
# (binary16 and fixed point share the 16-bit budget; fixed point, with 15
# fraction bits, is held to a tighter 5e-4 as well in the tests); 16-bit
# fixed-point links with FP32 vectors ("fx16l"): 5e-4, set by the links'
# 15 fraction bits
TOL_DSLASH = {"fp64": 1e-13, "fp32": 1e-6, "fp16": 5e-3, "fx16": 5e-3, "fx16l": 5e-4}
# double-float (FP64 data, FP32-pipe arithmetic with error-free transformations,
# about 48 significant bits) is held to the FP64 bound
TOL_DSLASH_DF = 1e-13


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


class Field:
    """A seeded gauge field held on the host (for the oracle) and the device."""

    _cache = {}

    def __init__(self, dims, eps, seed):
        self.dims = tuple(dims)
        self.fat, self.lng = synth.gauge_field(dims, eps, seed)
        self.fat_d = dev(self.fat)
        self.lng_d = dev(self.lng)

    @classmethod
    def get(cls, dims, eps=0.3, seed=1000):
        key = (tuple(dims), eps, seed)
        if key not in cls._cache:
            cls._cache.clear()
            cls._cache[key] = cls(dims, eps, seed)
        return cls._cache[key]

    def handle(self, recon=18, prec_mask=0):
        import paper_1712_00143_gb300 as stag

        return stag.stag_load_links(self.dims, self.fat_d, self.lng_d, recon_long=recon, prec_mask=prec_mask)


def oracle_true_residual(fat, lng, x, b, mass, dims, shift=0.0, chunk=1 << 21):
    """||b - (M + shift) x|| / ||b|| over the whole field with the oracle's
    operator, evaluated on chunks of output sites to bound host memory at
    48^3 x 96 (the same sums as oracle.true_residual)."""
    import oracle

    Vh = x.shape[0]
    t = np.empty_like(x)
    for s0 in range(0, Vh, chunk):
        idx = np.arange(s0, min(Vh, s0 + chunk))
        t[idx] = oracle.dslash(fat, lng, x, dims, 1, out_sites=idx)
    rr = 0.0
    for s0 in range(0, Vh, chunk):
        idx = np.arange(s0, min(Vh, s0 + chunk))
        mx = (mass * mass + shift) * x[idx] - oracle.dslash(fat, lng, t, dims, 0, out_sites=idx)
        rr += float(np.linalg.norm((b[idx] - mx).ravel()) ** 2)
    return float(np.sqrt(rr) / np.linalg.norm(b.ravel()))
