"""Helpers shared by the GPU parity tests: seeded fixtures on the device."""

import numpy as np
import pytest
import torch

import synth

requires_gpu = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")

# relative L2 error bounds: FP64 1e-13, FP32 1e-6, the 16-bit formats 5e-3
# (binary16 and fixed point share the 16-bit budget; fixed point, with 15
# fraction bits, is held to a tighter 5e-4 as well in the tests)
TOL_DSLASH = {"fp64": 1e-13, "fp32": 1e-6, "fp16": 5e-3, "fx16": 5e-3}


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
