"""Seeded synthetic inputs for the elastic Helmholtz solver.

This module generates problem data only: media (lambda, mu, rho), the
attenuation field gamma including the absorbing layer, the frequency omega,
point-source right-hand sides, and plain index re-layouts between the padded
device vector layout and the compact unknown ordering.  It holds none of the
method's arithmetic (no operator, preconditioner, multigrid or Krylov step),
so both the CPU oracle and the CUDA path may use it.

Problem statement followed (paper Sec. 4): a rectangular domain, point source
at the centre of the top edge, an absorbing layer of gradually increasing
attenuation on top of a natural attenuation gamma0 = 0.01*pi, and a frequency
giving about G_s grid points per shear wavelength in the slowest region.

Readings where the paper is silent (stated once here, used everywhere):
  * absorbing-layer profile: gamma = gamma0 + a * omega * (d / L)^2 with d the
    distance (in cells, from the cell centre) into the layer measured from its
    inner edge, maximised over axes and sides, L the layer width, and a = 0.2.
    The amplitude was calibrated on the paper's linear medium: with it the
    oracle's block-acoustic W(1,2) GMRES(5) counts at 400x128 (2/3/4 levels)
    land within a few percent of the printed 31/49/90 (Sec. 4.4, Table 4);
    a = 1 gives about half those counts;
  * grid spacing h = 1 / n_x (same h on every axis unless given), and
    omega = 2*pi*min(Vs) / (G_s * h);
  * the source is a vertical point force: the u2 (or u_d in d dimensions)
    face nearest the source point carries -1/(h1*h2[*h3]), the right-hand side
    being (-q; 0) as in the mixed system (Eq. 2.6).

Vector layout (device and C-ABI): padded, one array of shape
(d+1, n_d, ..., n_1) complex per vector, x_1 fastest.  Component k < d holds
u_{k+1} on the x_k-faces, indexed by the cell whose *lower* face it is; the
entries on the domain boundary (index 0 along axis k) are structural zeros
(normal displacement removed).  Component d holds p at cell centres.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA0 = 0.01 * math.pi
ABC_AMPLITUDE = 0.2


# ----------------------------------------------------------------------------
# elastic parameters
# ----------------------------------------------------------------------------
def vs_from_vp_nu(vp, nu):
    """Shear velocity from pressure velocity and Poisson ratio nu
    (nu = lambda / (2(lambda+mu)), Vp^2 = (lambda+2mu)/rho, Vs^2 = mu/rho)."""
    return vp * np.sqrt((1.0 - 2.0 * nu) / (2.0 - 2.0 * nu))


def lame_from_velocities(vp, vs, rho):
    """(lambda, mu) from (Vp, Vs, rho): mu = rho Vs^2, lambda = rho Vp^2 - 2 mu."""
    mu = rho * vs * vs
    lam = rho * vp * vp - 2.0 * mu
    return lam, mu


def omega_for(vs_min: float, h: float, gs: float = 10.0) -> float:
    """Angular frequency giving ``gs`` grid points per shear wavelength at the
    slowest shear velocity: lambda_s = 2 pi Vs / omega = gs * h."""
    return 2.0 * math.pi * vs_min / (gs * h)


# ----------------------------------------------------------------------------
# absorbing layer
# ----------------------------------------------------------------------------
def abc_gamma(shape, width: int, omega: float, gamma0: float = GAMMA0, amplitude: float = ABC_AMPLITUDE):
    """Attenuation field gamma on the cells of a grid of ``shape`` (numpy order,
    slowest axis first).  A layer of ``width`` cells on every side ramps
    quadratically from gamma0 at its inner edge to about
    gamma0 + amplitude * omega at the outer boundary."""
    d = np.zeros(shape, dtype=np.float64)
    if width > 0:
        for ax, n in enumerate(shape):
            s = np.arange(n, dtype=np.float64) + 0.5
            dist = np.maximum(np.maximum(width - s, 0.0), np.maximum(s - (n - width), 0.0))
            bshape = [1] * len(shape)
            bshape[ax] = n
            d = np.maximum(d, dist.reshape(bshape))
        d = d / float(width)
    return gamma0 + amplitude * omega * d * d


# ----------------------------------------------------------------------------
# media
# ----------------------------------------------------------------------------
@dataclass
class Problem:
    """One synthetic elastic Helmholtz problem (cell-centred arrays in numpy
    order, i.e. shape (n2, n1) in 2D and (n3, n2, n1) in 3D)."""
    name: str
    n: tuple            # cells along x1, x2[, x3]
    h: tuple            # spacing along x1, x2[, x3]
    lam: np.ndarray
    mu: np.ndarray
    rho: np.ndarray
    gamma: np.ndarray
    omega: float
    sources: list = field(default_factory=list)   # list of cell-index tuples (i1, i2[, i3]) of the u_d face
    meta: dict = field(default_factory=dict)

    @property
    def dim(self):
        return len(self.n)

    @property
    def shape(self):
        return tuple(reversed(self.n))


def _finish(name, n, h, vp, vs, rho, gs, abc, sources, meta, omega=None, gamma0=GAMMA0):
    lam, mu = lame_from_velocities(vp, vs, rho)
    if omega is None:
        omega = omega_for(float(vs.min()), float(min(h)), gs)
    gamma = abc_gamma(vp.shape, abc, omega, gamma0)
    meta = dict(meta)
    meta.update(gs=gs, abc=abc, omega=omega)
    return Problem(name, tuple(n), tuple(h), lam, mu, rho, gamma, float(omega), sources, meta)


def homogeneous(n1=64, n2=64, rho=1.0, vp=2.0, nu=0.25, gs=10.0, abc=8, source="centre"):
    """Constant medium (workload C1 at its defaults: 64x64, rho=1, Vp=2, nu=0.25)."""
    shape = (n2, n1)
    h = 1.0 / n1
    vpa = np.full(shape, vp)
    vsa = vs_from_vp_nu(vpa, nu)
    rhoa = np.full(shape, rho)
    src = [(n1 // 2, n2 // 2)] if source == "centre" else [(n1 // 2, max(abc, 1))]
    return _finish(f"homogeneous_{n1}x{n2}", (n1, n2), (h, h), vpa, vsa, rhoa, gs, abc, src,
                   dict(kind="homogeneous"))


def layered(n1=512, n2=512, nlayers=6, seed=2, vp_range=(1.5, 4.5), nu_range=(0.25, 0.45),
            gs=10.0, abc=20, nsrc=1, src_spacing=16):
    """Horizontal layers (boundaries at round(k*n2/nlayers)); per layer Vp and
    nu uniform in the given ranges, rho = 0.31 Vp^0.25 (workloads C2, C4)."""
    rng = np.random.default_rng(seed)
    vp_l = rng.uniform(*vp_range, size=nlayers)
    nu_l = rng.uniform(*nu_range, size=nlayers)
    bounds = [int(round(k * n2 / nlayers)) for k in range(nlayers + 1)]
    vp = np.empty((n2, n1))
    nu = np.empty((n2, n1))
    for k in range(nlayers):
        vp[bounds[k]:bounds[k + 1], :] = vp_l[k]
        nu[bounds[k]:bounds[k + 1], :] = nu_l[k]
    vs = vs_from_vp_nu(vp, nu)
    rho = 0.31 * vp ** 0.25
    h = 1.0 / n1
    zs = max(abc, 1)
    if nsrc == 1:
        src = [(n1 // 2, zs)]
    else:
        src = [(src_spacing // 2 + k * src_spacing, zs) for k in range(nsrc)]
    return _finish(f"layered_{n1}x{n2}", (n1, n2), (h, h), vp, vs, rho, gs, abc, src,
                   dict(kind="layered", seed=seed, vp_layers=vp_l.tolist(), nu_layers=nu_l.tolist()))


def gaussian_random_field(shape, corr_len, seed):
    """Zero-mean, unit-std stationary field: white noise convolved (periodic,
    via FFT) with a Gaussian kernel of standard deviation corr_len/sqrt(2)."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(shape)
    sig = corr_len / math.sqrt(2.0)
    kern_hat = np.ones(shape)
    for ax, n in enumerate(shape):
        k = np.fft.fftfreq(n) * 2.0 * math.pi
        g = np.exp(-0.5 * (sig * k) ** 2)
        bshape = [1] * len(shape)
        bshape[ax] = n
        kern_hat = kern_hat * g.reshape(bshape)
    f = np.real(np.fft.ifftn(np.fft.fftn(w) * kern_hat))
    f = f - f.mean()
    return f / f.std()


def _std_normal_cdf(x):
    from scipy.special import ndtr
    return ndtr(x)


def grf_medium(n=(1024, 1024), corr=32.0, seed_vp=3, seed_nu=4, gs=10.0, abc=20,
               log_vp_mean=math.log(3.0), log_vp_std=0.2, nu_lo=0.3, nu_hi=0.49):
    """Smooth random medium: log Vp a Gaussian random field (mean log 3, std
    0.2), nu = 0.3 + 0.19 Phi(g2) from an independent field, rho = 0.31
    Vp^0.25 (workloads C3, C5)."""
    shape = tuple(reversed(n))
    g1 = gaussian_random_field(shape, corr, seed_vp)
    g2 = gaussian_random_field(shape, corr, seed_nu)
    vp = np.exp(log_vp_mean + log_vp_std * g1)
    nu = nu_lo + (nu_hi - nu_lo) * _std_normal_cdf(g2)
    vs = vs_from_vp_nu(vp, nu)
    rho = 0.31 * vp ** 0.25
    h = 1.0 / n[0]
    src = [tuple([n[0] // 2] + [n[k] // 2 for k in range(1, len(n) - 1)] + [max(abc, 1)])]
    return _finish(f"grf_{'x'.join(map(str, n))}", tuple(n), tuple([h] * len(n)), vp, vs, rho, gs,
                   abc, src, dict(kind="grf", corr=corr, seeds=(seed_vp, seed_nu)))


def linear_medium(n1=200, n2=64, omega=1.75 * math.pi, lam_factor=1.0, abc=20,
                  width=16.0, depth=5.0):
    """The paper's linear model (Sec. 4): a 16 km x 5 km domain whose rho,
    mu and lambda vary linearly with depth over rho in [2,3], mu in [1,15],
    lambda in [4,20] (lambda optionally multiplied by ``lam_factor``)."""
    h1 = width / n1
    h2 = depth / n2
    z = (np.arange(n2) + 0.5) / n2
    col = lambda a, b: np.repeat((a + (b - a) * z)[:, None], n1, axis=1)
    rho = col(2.0, 3.0)
    mu = col(1.0, 15.0)
    lam = col(4.0, 20.0) * lam_factor
    gamma = abc_gamma((n2, n1), abc, omega)
    src = [(n1 // 2, max(abc, 1))]
    return Problem(f"linear_{n1}x{n2}", (n1, n2), (h1, h2), lam, mu, rho, gamma, float(omega), src,
                   dict(kind="linear", lam_factor=lam_factor, abc=abc))


def random_medium(n, seed, lam_range=(1.0, 4.0), mu_range=(0.5, 2.0), rho_range=(0.8, 1.5),
                  omega=None, abc=2, h=None):
    """Rough, cell-wise i.i.d. medium for parity tests on small grids."""
    rng = np.random.default_rng(seed)
    shape = tuple(reversed(n))
    lam = rng.uniform(*lam_range, size=shape)
    mu = rng.uniform(*mu_range, size=shape)
    rho = rng.uniform(*rho_range, size=shape)
    if h is None:
        h = tuple([1.0 / n[0]] * len(n))
    vs = np.sqrt(mu / rho)
    if omega is None:
        omega = omega_for(float(vs.min()), float(min(h)), 10.0)
    gamma = abc_gamma(shape, abc, omega)
    src = [tuple([n[0] // 2] + [n[k] // 2 for k in range(1, len(n))])]
    return Problem(f"random_{'x'.join(map(str, n))}_s{seed}", tuple(n), tuple(h), lam, mu, rho,
                   gamma, float(omega), src, dict(kind="random", seed=seed))


# ----------------------------------------------------------------------------
# standard workloads
# ----------------------------------------------------------------------------
def config(name: str) -> Problem:
    """The five named workloads c1 .. c5, and c5s, a 64^3 copy of c5."""
    if name == "c1":
        return homogeneous(64, 64, 1.0, 2.0, 0.25, 10.0, 8, "centre")
    if name == "c2":
        return layered(512, 512, 6, 2)
    if name == "c3":
        return grf_medium((1024, 1024), 32.0, 3, 4, 10.0, 20)
    if name == "c4":
        return layered(1024, 512, 6, 5, nsrc=64, src_spacing=16)
    if name == "c5":
        return grf_medium((128, 128, 128), 16.0, 3, 4, 8.0, 10)
    if name == "c5s":
        # the c5 medium on a 64^3 grid (correlation length and absorbing layer
        # halved): a small case of the 3-D kernels for profiling
        return grf_medium((64, 64, 64), 8.0, 3, 4, 8.0, 5)
    raise KeyError(name)


# ----------------------------------------------------------------------------
# layouts and right-hand sides (pure index re-arrangement)
# ----------------------------------------------------------------------------
def padded_shape(n):
    """Shape of one padded vector: (d+1, n_d, ..., n_1)."""
    return (len(n) + 1,) + tuple(reversed(n))


def _face_slices(d, k):
    """numpy slice selecting the unknowns of component k (faces with index >= 1
    along axis k) inside one (n_d..n_1) array."""
    sl = [slice(None)] * d
    sl[d - 1 - k] = slice(1, None)
    return tuple(sl)


def compact_sizes(n):
    """Numbers of unknowns per component [u_1 .. u_d, p] in the compact order."""
    d = len(n)
    tot = int(np.prod(n))
    sizes = [tot // n[k] * (n[k] - 1) for k in range(d)]
    return sizes + [tot]


def padded_to_compact(v, n):
    """Padded (d+1, n_d..n_1) -> compact 1-D vector [u_1 | .. | u_d | p], each
    component x_1-fastest over its unknowns only."""
    d = len(n)
    v = np.asarray(v)
    parts = [v[k][_face_slices(d, k)].ravel() for k in range(d)]
    parts.append(v[d].ravel())
    return np.concatenate(parts)


def compact_to_padded(c, n, dtype=np.complex128):
    """Inverse of padded_to_compact; boundary-normal entries set to zero."""
    d = len(n)
    out = np.zeros(padded_shape(n), dtype=dtype)
    off = 0
    shp = tuple(reversed(n))
    for k in range(d):
        sub = list(shp)
        sub[d - 1 - k] -= 1
        cnt = int(np.prod(sub))
        out[k][_face_slices(d, k)] = np.asarray(c[off:off + cnt]).reshape(sub)
        off += cnt
    out[d] = np.asarray(c[off:off + int(np.prod(shp))]).reshape(shp)
    return out


def point_source(prob: Problem, src=None, amplitude=1.0):
    """Padded right-hand side (-q; 0) for a vertical point force on the u_d face
    at cell index ``src`` (the face below that cell along x_d)."""
    n = prob.n
    d = len(n)
    if src is None:
        src = prob.sources[0]
    b = np.zeros(padded_shape(n), dtype=np.complex128)
    idx = list(reversed(src))
    idx[0] = min(max(idx[0], 1), n[d - 1] - 1)   # u_d face index along x_d must be interior
    b[d - 1][tuple(idx)] = -amplitude / float(np.prod(prob.h))
    return b


def all_sources(prob: Problem):
    """Stacked padded right-hand sides, one per source in ``prob.sources``."""
    return np.stack([point_source(prob, s) for s in prob.sources])


def random_vector(n, seed, dtype=np.complex128):
    """Seeded random padded vector with zero boundary-normal entries."""
    rng = np.random.default_rng(seed)
    v = (rng.standard_normal(padded_shape(n)) + 1j * rng.standard_normal(padded_shape(n))).astype(dtype)
    d = len(n)
    for k in range(d):
        sl = [slice(None)] * d
        sl[d - 1 - k] = 0
        v[k][tuple(sl)] = 0
    return v
