"""Seeded gauge fields and sources in the canonical layout.

Canonical layout (the only one callers of the library see):
  * sites are lexicographic with x fastest, ``lex = x + Lx*(y + Ly*(z + Lz*t))``;
  * a link field is ``[V][mu][3][3]`` complex128, mu = x, y, z, t, row-major
    colour matrices; ``field[lex, mu]`` is the link from site lex to lex + mu;
  * a single-parity colour-vector field is ``[V/2][3]`` complex128 indexed by
    ``lex // 2`` (all extents are even, so this is one-to-one per parity).

Recipe of the benchmark workloads (staggered multi-shift / single-mass CG of
Sec. 4.1 on synthetic stand-ins for the paper's equilibrated ensembles):
  * thin links U = exp(i*eps*H), H a random traceless Hermitian 3x3 matrix
    with complex N(0,1) entries before symmetrisation, reunitarised to SU(3);
  * fat link F_mu = U_mu + (1/8) * (sum of the six three-link staples around
    mu, two for each nu != mu);
  * long (Naik) link L_mu(x) = -(1/24) U_mu(x) U_mu(x+mu) U_mu(x+2mu);
  * periodic boundaries; no staggered phases here (they belong to the
    operator, not to the field).

Heavy batched 3x3 products run on PyTorch CPU tensors (multi-threaded);
random numbers come from :mod:`synth.rng`.
"""

from dataclasses import dataclass

import numpy as np
import torch

from .rng import counter_normals

# Stream identifiers that keep the variates of different fields apart.
STREAM_THIN = 1
STREAM_SOURCE = 2
STREAM_GAUGE_TRANSFORM = 3
STREAM_SPINOR = 4


@dataclass(frozen=True)
class Lattice:
    """A 4-d periodic lattice with even extents (Lx, Ly, Lz, Lt)."""

    dims: tuple

    def __post_init__(self):
        d = tuple(int(v) for v in self.dims)
        if len(d) != 4 or any(v < 2 or v % 2 for v in d):
            raise ValueError(f"extents must be 4 even numbers >= 2, got {self.dims}")
        object.__setattr__(self, "dims", d)

    @property
    def V(self):
        Lx, Ly, Lz, Lt = self.dims
        return Lx * Ly * Lz * Lt

    @property
    def Vh(self):
        return self.V // 2

    @property
    def shape_tzyx(self):
        """Site-array shape with t slowest, x fastest (matches lex order)."""
        Lx, Ly, Lz, Lt = self.dims
        return (Lt, Lz, Ly, Lx)


# axis of the (t, z, y, x) site array along which direction mu runs
_AXIS = {0: 3, 1: 2, 2: 1, 3: 0}


def _shift(a, mu, k):
    """Field value at x + k*mu (periodic), for a (Lt, Lz, Ly, Lx, ...) tensor."""
    return torch.roll(a, shifts=-k, dims=_AXIS[mu])


def _dag(a):
    return a.conj().transpose(-1, -2)


def _reunitarise(u):
    """Gram-Schmidt on rows 0 and 1, row 2 = conj(row0 x row1): an SU(3) matrix."""
    r0 = u[..., 0, :]
    r0 = r0 / torch.linalg.vector_norm(r0, dim=-1, keepdim=True)
    r1 = u[..., 1, :]
    r1 = r1 - (r0.conj() * r1).sum(-1, keepdim=True) * r0
    r1 = r1 / torch.linalg.vector_norm(r1, dim=-1, keepdim=True)
    r2 = torch.linalg.cross(r0, r1, dim=-1).conj()
    return torch.stack([r0, r1, r2], dim=-2)


def random_su3(n, eps, seed, stream, offset=0):
    """``n`` SU(3) matrices exp(i*eps*H), H traceless Hermitian, reunitarised.

    Matrix j uses the normals with counters (offset + j)*18 .. +17, so any
    sub-range can be regenerated independently.
    """
    g = counter_normals_range(seed, stream, 18 * offset, 18 * n).reshape(n, 3, 3, 2)
    a = torch.from_numpy(g[..., 0] + 1j * g[..., 1])
    h = 0.5 * (a + _dag(a))
    tr = torch.diagonal(h, dim1=-2, dim2=-1).sum(-1) / 3.0
    h = h - tr[:, None, None] * torch.eye(3, dtype=h.dtype)
    u = torch.linalg.matrix_exp((1j * eps) * h)
    return _reunitarise(u)


def counter_normals_range(seed, stream, start, count):
    """Normals with counters start .. start+count-1 (start must be even)."""
    if start % 2:
        raise ValueError("start must be even")
    if start == 0:
        return counter_normals(seed, stream, count)
    from .rng import counter_uniforms

    npairs = (count + 1) // 2
    u = counter_uniforms(seed, stream, start, 2 * npairs)
    rad = np.sqrt(-2.0 * np.log(u[0::2]))
    ang = (2.0 * np.pi) * u[1::2]
    out = np.empty(2 * npairs)
    out[0::2] = rad * np.cos(ang)
    out[1::2] = rad * np.sin(ang)
    return out[:count]


def thin_links(lat, eps, seed):
    """SU(3) thin links as a (Lt, Lz, Ly, Lx, 4, 3, 3) complex128 tensor."""
    n = 4 * lat.V
    chunk = 1 << 21
    parts = [random_su3(min(chunk, n - s), eps, seed, STREAM_THIN, offset=s) for s in range(0, n, chunk)]
    return torch.cat(parts).reshape(*lat.shape_tzyx, 4, 3, 3)


def fat_links(u):
    """F_mu(x) = U_mu(x) + 1/8 sum_{nu != mu} [S+_{mu nu}(x) + S-_{mu nu}(x)].

    S+_{mu nu}(x) = U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag         (upper staple)
    S-_{mu nu}(x) = U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu)    (lower staple)
    """
    out = torch.empty_like(u)
    for mu in range(4):
        umu = u[..., mu, :, :]
        acc = umu.clone()
        for nu in range(4):
            if nu == mu:
                continue
            unu = u[..., nu, :, :]
            up = unu @ _shift(umu, nu, 1) @ _dag(_shift(unu, mu, 1))
            unu_m = _shift(unu, nu, -1)
            dn = _dag(unu_m) @ _shift(umu, nu, -1) @ _shift(_shift(unu, nu, -1), mu, 1)
            acc += 0.125 * (up + dn)
        out[..., mu, :, :] = acc
    return out


def naik_links(u, coeff=-1.0 / 24.0):
    """L_mu(x) = coeff * U_mu(x) U_mu(x+mu) U_mu(x+2mu)."""
    out = torch.empty_like(u)
    for mu in range(4):
        umu = u[..., mu, :, :]
        out[..., mu, :, :] = coeff * (umu @ _shift(umu, mu, 1) @ _shift(umu, mu, 2))
    return out


def gauge_field(dims, eps, seed, return_thin=False):
    """(fat, long) canonical [V][4][3][3] complex128 numpy arrays for one seed."""
    lat = Lattice(tuple(dims))
    u = thin_links(lat, eps, seed)
    fat = fat_links(u).reshape(lat.V, 4, 3, 3).numpy()
    lng = naik_links(u).reshape(lat.V, 4, 3, 3).numpy()
    if return_thin:
        return fat, lng, u.reshape(lat.V, 4, 3, 3).numpy()
    return fat, lng


def links_from_thin(dims, thin):
    """(fat, long) canonical arrays from given thin links [V][4][3][3]."""
    lat = Lattice(tuple(dims))
    u = torch.from_numpy(np.ascontiguousarray(thin)).reshape(*lat.shape_tzyx, 4, 3, 3)
    return (
        fat_links(u).reshape(lat.V, 4, 3, 3).numpy(),
        naik_links(u).reshape(lat.V, 4, 3, 3).numpy(),
    )


def gaussian_source(dims, seed, nrhs=None, stream=STREAM_SOURCE):
    """Single-parity source(s): [Vh][3] (or [nrhs][Vh][3]) complex128, N(0,1) re/im."""
    lat = Lattice(tuple(dims))
    n = lat.Vh * 3 * (1 if nrhs is None else nrhs)
    g = counter_normals(seed, stream, 2 * n).reshape(-1, 2)
    v = g[:, 0] + 1j * g[:, 1]
    return v.reshape(lat.Vh, 3) if nrhs is None else v.reshape(nrhs, lat.Vh, 3)


def random_spinor(dims, seed, full=False):
    """Random colour-vector field on one parity ([Vh][3]) or all sites ([V][3])."""
    lat = Lattice(tuple(dims))
    n = (lat.V if full else lat.Vh) * 3
    g = counter_normals(seed, STREAM_SPINOR, 2 * n).reshape(-1, 2)
    return (g[:, 0] + 1j * g[:, 1]).reshape(-1, 3)


def random_gauge_transform(dims, seed, eps=2.0):
    """One SU(3) matrix per site, [V][3][3] complex128."""
    lat = Lattice(tuple(dims))
    return random_su3(lat.V, eps, seed, STREAM_GAUGE_TRANSFORM).numpy()


def gauge_transform_links(dims, thin, g):
    """U'_mu(x) = G(x) U_mu(x) G(x+mu)^dag on canonical [V][4][3][3] thin links."""
    lat = Lattice(tuple(dims))
    u = torch.from_numpy(np.ascontiguousarray(thin)).reshape(*lat.shape_tzyx, 4, 3, 3)
    gg = torch.from_numpy(np.ascontiguousarray(g)).reshape(*lat.shape_tzyx, 3, 3)
    out = torch.empty_like(u)
    for mu in range(4):
        out[..., mu, :, :] = gg @ u[..., mu, :, :] @ _dag(_shift(gg, mu, 1))
    return out.reshape(lat.V, 4, 3, 3).numpy()
