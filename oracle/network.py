"""FP64 oracle of the gauge-covariant network used as a CG preconditioner (test infrastructure).

The network maps a residual field to an approximation of the error field it
came from (e = M^{-1} r).  It is built only from operations that commute with
gauge transformations G(x) -- parallel transport by the fat links and
colour-blind channel mixing -- so N(G r) = G N(r) (pinned by a test).

Fields live on the full lattice as [C][V][3] complex128 (C channels, lex
site order, colour).  Directions d = 0..8 of a layer:
    d = 0          (T_0 h)(x) = h(x)
    d = 1 + 2 mu   (T_d h)(x) =  1/2 eta_mu(x) F_mu(x) h(x + mu)
    d = 2 + 2 mu   (T_d h)(x) = -1/2 eta_mu(x) F_mu(x - mu)^dag h(x - mu)
i.e. the fat-link hops of the staggered operator itself (sum over d != 0 of
T_d is D without its Naik terms); the staggered phases are a fixed sign
field, so the transports stay gauge covariant.  (T_{1+2mu})^dag =
-T_{2+2mu}.  A layer with real weights W[d][c][c'] computes
    pre_c(x) = sum_d sum_c' W[d][c][c'] (T_d h_c')(x)
and a hidden layer applies the covariant gate
    sigma_c(v)(x) = v(x) * s,   s = 1 / (1 + exp(-(|v(x)|^2 - b_c)))
(|v(x)|^2 summed over colour is gauge invariant).  The last layer is linear.
Channels 1 -> 16 -> 16 -> 16 -> 1 in the benchmark workload.

Input and output: an even-site residual r ([Vh][3]) is scaled to unit
mean-square per site, r_hat = r * sqrt(Vh) / ||r||, placed on the even sites
of a one-channel field (zeros on odd sites); the prediction is the even-site
part of the output channel, and z = N(r) = prediction * ||r|| / sqrt(Vh).

Two training losses, both on the scaled fields:
    error space     L_e = ||z_hat - e_hat||^2 / ||e_hat||^2
    residual space  L_r = ||M z_hat - r_hat||^2 / ||r_hat||^2
with M = m^2 - D_eo D_oe the even-odd operator of the pair's gauge field and
mass.  Since r = M e, L_r = ||M (z_hat - e_hat)||^2 / ||M e_hat||^2: the
error weighted by M^2, which stresses the high modes a network of a few
nearest-neighbour hops can represent; L_e is dominated by the low modes that
make up most of e at small mass.

Gradients use the convention G = dL/dRe + i dL/dIm for complex fields, so a
linear map y = A h has G_h = A^dag G_y.

Parity status: forward, backward and both losses are pinned by finite
differences of the loss in FP64 and by gauge covariance; the restriction of
the forward pass to sampled output sites is pinned by the whole-field forward
(tests/test_network_oracle.py).
"""

import numpy as np

from . import staggered

NDIR = 9


def _site_roll(a, dims, mu, k, site_axis):
    """Values at x + k*mu (periodic) of an array whose axis `site_axis` runs over lex sites."""
    Lx, Ly, Lz, Lt = dims
    shp = a.shape
    b = a.reshape(shp[:site_axis] + (Lt, Lz, Ly, Lx) + shp[site_axis + 1 :])
    ax = site_axis + {0: 3, 1: 2, 2: 1, 3: 0}[mu]
    return np.roll(b, -k, axis=ax).reshape(shp)


def _eta(dims, mu):
    """eta_mu(x) for every lex site: 1, (-1)^x, (-1)^(x+y), (-1)^(x+y+z)."""
    Lx, Ly, Lz, Lt = dims
    lex = np.arange(Lx * Ly * Lz * Lt)
    c = [lex % Lx, (lex // Lx) % Ly, (lex // (Lx * Ly)) % Lz]
    s = sum(c[:mu]) if mu > 0 else np.zeros_like(lex)
    return np.where(s % 2 == 0, 1.0, -1.0)


def transport(fat, h, dims, d):
    """(T_d h) for a [C, V, 3] field."""
    if d == 0:
        return h.copy()
    mu = (d - 1) // 2
    eta = _eta(dims, mu)[None, :, None]
    if d % 2 == 1:  # +1/2 eta F_mu(x) h(x + mu)
        return 0.5 * eta * np.einsum("vij,cvj->cvi", fat[:, mu], _site_roll(h, dims, mu, +1, 1))
    # -1/2 eta F_mu(x - mu)^dag h(x - mu)
    Fm = _site_roll(fat[:, mu], dims, mu, -1, 0)
    return -0.5 * eta * np.einsum("vji,cvj->cvi", np.conj(Fm), _site_roll(h, dims, mu, -1, 1))


def transport_adjoint(fat, g, dims, d):
    """(T_d^dag g): T_0 is self-adjoint and (T_{1+2mu})^dag = -T_{2+2mu}."""
    if d == 0:
        return g.copy()
    return -transport(fat, g, dims, d + 1 if d % 2 == 1 else d - 1)


def gate(v, b):
    """v * sigmoid(|v|^2 - b_c) per channel c and site; returns (out, s)."""
    n2 = (np.abs(v) ** 2).sum(axis=-1)  # [C, V]
    s = 1.0 / (1.0 + np.exp(-(n2 - b[:, None])))
    return v * s[..., None], s


def layer_forward(fat, W, h, dims):
    """pre[c] = sum_d sum_c' W[d, c, c'] T_d h[c']."""
    pre = np.zeros((W.shape[1],) + h.shape[1:], dtype=np.complex128)
    for d in range(NDIR):
        th = transport(fat, h, dims, d)
        pre += np.einsum("ab,bvi->avi", W[d], th)
    return pre


def forward(fat, params, r, dims, parity_sites):
    """Network output for an even-site residual r; returns (z, cache).

    params: list of (W [9, Cout, Cin] float64, b [Cout] float64 or None).
    parity_sites: lex indices of the even sites in checkerboard order.
    """
    V = fat.shape[0]
    Vh = len(parity_sites)
    nr = np.linalg.norm(r)
    scale = np.sqrt(Vh) / nr
    h = np.zeros((1, V, 3), dtype=np.complex128)
    h[0, parity_sites] = r * scale
    cache = {"h": [h], "pre": [], "s": [], "scale": scale}
    for li, (W, b) in enumerate(params):
        pre = layer_forward(fat, W, h, dims)
        cache["pre"].append(pre)
        if b is not None:
            h, s = gate(pre, b)
            cache["s"].append(s)
        else:
            h = pre
            cache["s"].append(None)
        cache["h"].append(h)
    pred = h[0, parity_sites]
    return pred / scale, cache


def forward_at_sites(fat, params, r, dims, parity_sites, out_sites):
    """The even-site output z = N(r) at checkerboard indices ``out_sites`` only.

    The same definition as :func:`forward`, restricted to what those outputs
    read: a layer's output at x depends on its input at x and x +- mu, so with
    L layers left the input is needed on the sites within L hops of the
    requested ones.  The site sets S_L (the requested sites) and S_{k-1} =
    S_k and its neighbours are built first; layer k is evaluated on S_{k+1}
    from its input on S_k.  The input scale sqrt(Vh)/||r|| is the global one.
    Returns a [len(out_sites)][3] array in the order of ``out_sites``.
    """
    dims = tuple(dims)
    nl = len(params)
    Vh = len(parity_sites)
    scale = np.sqrt(Vh) / np.linalg.norm(r)
    targets = np.asarray(parity_sites)[np.asarray(out_sites, dtype=np.int64)]
    sets = [None] * (nl + 1)
    sets[nl] = np.unique(targets)
    for k in range(nl, 0, -1):
        c = staggered.site_coords(dims, sets[k])
        nb = [sets[k]] + [staggered.neighbour_lex(dims, c, mu, s) for mu in range(4) for s in (1, -1)]
        sets[k - 1] = np.unique(np.concatenate(nb))
    lex0 = sets[0]
    c0 = staggered.site_coords(dims, lex0)
    even = c0.sum(axis=1) % 2 == 0
    h = np.zeros((1, len(lex0), 3), dtype=np.complex128)
    h[0, even] = r[lex0[even] // 2] * scale
    for k, (W, b) in enumerate(params):
        X, Y = sets[k + 1], sets[k]
        cX = staggered.site_coords(dims, X)
        pre = np.zeros((W.shape[1], len(X), 3), dtype=np.complex128)
        for d in range(NDIR):
            pre += np.einsum("ab,bvi->avi", W[d], _transport_on(fat, h, Y, X, cX, dims, d))
        h = gate(pre, b)[0] if b is not None else pre
    return h[0, np.searchsorted(sets[nl], targets)] / scale


def _transport_on(fat, h, Y, X, cX, dims, d):
    """(T_d h) on the sorted lex sites X, for h given on the sorted lex sites Y
    (Y holds X and its +-mu neighbours)."""
    if d == 0:
        return h[:, np.searchsorted(Y, X)]
    mu = (d - 1) // 2
    eta = staggered.staggered_phase(mu, cX)[None, :, None]
    if d % 2 == 1:  # +1/2 eta F_mu(x) h(x + mu)
        nb = staggered.neighbour_lex(dims, cX, mu, +1)
        return 0.5 * eta * np.einsum("vij,cvj->cvi", fat[X, mu], h[:, np.searchsorted(Y, nb)])
    nb = staggered.neighbour_lex(dims, cX, mu, -1)  # -1/2 eta F_mu(x - mu)^dag h(x - mu)
    return -0.5 * eta * np.einsum("vji,cvj->cvi", np.conj(fat[nb, mu]), h[:, np.searchsorted(Y, nb)])


def loss(fat, params, r, e, dims, parity_sites):
    """||N_hat(r_hat) - e_hat||^2 / ||e_hat||^2 with both sides scaled by sqrt(Vh)/||r||."""
    z, cache = forward(fat, params, r, dims, parity_sites)
    diff = (z - e) * cache["scale"]
    ne2 = np.linalg.norm(e * cache["scale"]) ** 2
    return float(np.linalg.norm(diff) ** 2 / ne2), cache


def backward_from(fat, params, cache, g_pred, dims, parity_sites):
    """Gradients of a loss whose derivative with respect to the scaled even-site
    prediction z_hat is g_pred ([Vh][3]); returns a list of (dW, db)."""
    V = fat.shape[0]
    g = np.zeros((1, V, 3), dtype=np.complex128)
    g[0, parity_sites] = g_pred
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, b = params[li]
        pre = cache["pre"][li]
        hin = cache["h"][li]
        db = None
        if b is not None:
            s = cache["s"][li]
            sp = s * (1.0 - s)
            proj = np.real((np.conj(g) * pre).sum(axis=-1))  # Re<G_out, v> per channel, site
            db = -(proj * sp).sum(axis=1)
            g = g * s[..., None] + (2.0 * sp * proj)[..., None] * pre
        dW = np.zeros_like(W)
        gin = np.zeros_like(hin)
        for d in range(NDIR):
            th = transport(fat, hin, dims, d)
            dW[d] = np.real(np.einsum("avi,bvi->ab", np.conj(g), th))
            gin += transport_adjoint(fat, np.einsum("ab,avi->bvi", W[d], g), dims, d)
        grads[li] = (dW, db)
        g = gin
    return grads


def backward(fat, params, r, e, dims, parity_sites):
    """(L_e, grads) with grads a list of (dW, db) matching params."""
    L, cache = loss(fat, params, r, e, dims, parity_sites)
    ehat = e * cache["scale"]
    pred = cache["h"][-1][0, parity_sites]
    g_pred = 2.0 * (pred - ehat) / (np.linalg.norm(ehat) ** 2)
    return L, backward_from(fat, params, cache, g_pred, dims, parity_sites)


def loss_residual(fat, lng, params, r, mass, dims, parity_sites):
    """L_r = ||M z_hat - r_hat||^2 / ||r_hat||^2 with M = m^2 - D_eo D_oe."""
    z, cache = forward(fat, params, r, dims, parity_sites)
    zhat = cache["h"][-1][0, parity_sites]
    rhat = r * cache["scale"]
    diff = staggered.apply_m(fat, lng, zhat, mass, dims) - rhat
    cache["resid_diff"] = diff
    return float(np.linalg.norm(diff) ** 2 / np.linalg.norm(rhat) ** 2), cache


def backward_residual(fat, lng, params, r, mass, dims, parity_sites):
    """(L_r, grads): dL_r/dz_hat = 2 M (M z_hat - r_hat) / ||r_hat||^2 (M is Hermitian)."""
    L, cache = loss_residual(fat, lng, params, r, mass, dims, parity_sites)
    rhat = r * cache["scale"]
    g_pred = 2.0 * staggered.apply_m(fat, lng, cache["resid_diff"], mass, dims) / np.linalg.norm(rhat) ** 2
    return L, backward_from(fat, params, cache, g_pred, dims, parity_sites)


def init_params(channels, seed):
    """Seeded initial weights (scaled normal, rounded to bfloat16) and zero biases."""
    rng = np.random.default_rng(seed)
    params = []
    for li in range(len(channels) - 1):
        cin, cout = channels[li], channels[li + 1]
        W = rng.normal(0.0, 1.0 / np.sqrt(NDIR * cin), size=(NDIR, cout, cin))
        W[0] += np.eye(cout, cin) * 0.5
        b = np.zeros(cout) if li < len(channels) - 2 else None
        params.append((bf16_round(W), b))
    return params


def bf16_round(a):
    """Round float64 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
