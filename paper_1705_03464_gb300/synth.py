"""Seeded synthetic galaxy catalogues (inputs only).

This module draws the inputs that both the CUDA path and the FP64 oracle
consume. It holds none of the estimator's arithmetic: no pair finding,
no mass assignment, no correlation. The paper measures on Abacus N-body
boxes with FoF halos (Sec. 3.1), which are not available here; these
catalogues stand in for them with the same structure:

* halos Poisson-sampled from a lognormal density field on a 64^3 grid whose
  Gaussian part has P(k) ~ k^-1.5 and unit log-variance;
* halo masses drawn from dn/dlnM ~ M^-0.9 exp(-M / 10^14.5) on
  [10^12.5, 10^15] Msun/h;
* galaxies from the five-parameter HOD of Sec. 3.3 (eq. hod): centrals at the
  halo centre with probability <n_cen>, Poisson satellites with mean <n_sat>,
  placed uniformly in a sphere of radius 1.6 (M/1e15)^(1/3) Mpc/h (the
  paper places satellites on halo particles, which do not exist here);
* velocities: a Gaussian 300 km/s per axis for the halo, plus an isotropic
  Gaussian of dispersion sqrt(G M / 2R) per axis for satellites.

Random numbers come from NumPy's PCG64 seeded with the caller's seed. The
halo density is set so that the expected galaxy count equals the requested
one (the HOD integrated over the mass function).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

# Gravitational constant in Mpc (km/s)^2 / Msun.
G_NEWTON = 4.301e-9
# Z09 design of the HOD (Sec. 3.3): log10 Mcut, log10 M1, sigma, alpha, kappa.
HOD_Z09 = (13.35, 13.8, 0.85, 1.0, 1.0)
# Mpc/h per km/s for the RSD shift x' = x + v / H(z) (eq. RSD) at z = 0.5 in
# flat LCDM with Omega_m = 0.31: (1 + z) / (100 E(z)).
RSD_FACTOR_Z05 = (1.5) / (100.0 * math.sqrt(0.31 * 1.5 ** 3 + 0.69))


@dataclasses.dataclass
class Workload:
    """One synthetic workload: box, mesh, binning and catalogue size."""
    name: str
    box_L: float
    mesh_n: int
    assign: int              # 0 = NGP, 1 = CIC
    n_gal: int               # target galaxy count
    s_edges: tuple
    n_mu: int
    r_edges: tuple
    n_mur: int
    rsd: bool
    precision: int           # 0 = FP32 batched FFT, 1 = FP64 per bin
    bins_per_batch: int = 0
    r_perp_cut: float = 0.0

    @property
    def rsd_factor(self) -> float:
        return RSD_FACTOR_Z05 if self.rsd else 0.0


def _edges(lo, hi, n):
    return tuple(float(x) for x in np.linspace(lo, hi, n + 1))


# The workloads of the benchmark suite, named by what they are.
WORKLOADS = {
    # real space, 128^3 NGP, ~1.2k galaxies, FP64 path
    "real_ngp_128": Workload("real_ngp_128", 128.0, 128, 0, 1200,
                             _edges(0, 8, 8), 1, _edges(8, 40, 8), 1,
                             False, 1),
    # real + redshift space, 512^3 CIC, ~40k galaxies, FP32 FFT
    "rsd_cic_512": Workload("rsd_cic_512", 512.0, 512, 1, 40000,
                            _edges(0, 10, 10), 5, _edges(10, 60, 10), 5,
                            True, 0),
    # paper-scale box: L = 1100 Mpc/h, 1024^3 CIC, n = 3e-4 (h/Mpc)^3
    "paper_1024": Workload("paper_1024", 1100.0, 1024, 1,
                           int(round(3e-4 * 1100.0 ** 3)),
                           _edges(0, 10, 20), 5, _edges(10, 60, 10), 5,
                           False, 0, 16),
}


def hod_mean_occupation(M, hod=HOD_Z09):
    """<n_cen>, <n_sat> of eq. hod for halo masses M (Msun/h), natural log."""
    from scipy.special import erfc
    log_mcut, log_m1, sigma, alpha, kappa = hod
    mcut = 10.0 ** log_mcut
    m1 = 10.0 ** log_m1
    ncen = 0.5 * erfc(np.log(mcut / M) / (math.sqrt(2.0) * sigma))
    x = np.clip((M - kappa * mcut) / m1, 0.0, None)
    nsat = np.where(M > kappa * mcut, x ** alpha, 0.0)
    return ncen, nsat


def _mass_grid():
    lnm = np.linspace(12.5 * math.log(10), 15.0 * math.log(10), 4097)
    M = np.exp(lnm)
    dn = M ** -0.9 * np.exp(-M / 10.0 ** 14.5)
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (dn[1:] + dn[:-1]) * np.diff(lnm))])
    return lnm, M, dn, cdf / cdf[-1]


def _mean_gal_per_halo(hod):
    lnm, M, dn, _ = _mass_grid()
    ncen, nsat = hod_mean_occupation(M, hod)
    w = dn / np.trapezoid(dn, lnm)
    return float(np.trapezoid(w * (ncen + nsat), lnm))


def _lognormal_field(rng, ng=64):
    """1 + delta on an ng^3 grid; ln(1+delta) Gaussian, P(k) ~ k^-1.5, var 1."""
    white = rng.standard_normal((ng, ng, ng))
    f = np.fft.rfftn(white)
    kx = np.fft.fftfreq(ng)[:, None, None]
    ky = np.fft.fftfreq(ng)[None, :, None]
    kz = np.fft.rfftfreq(ng)[None, None, :]
    k = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.zeros_like(k)
    amp[k > 0] = k[k > 0] ** (-0.75)
    g = np.fft.irfftn(f * amp, s=(ng, ng, ng), axes=(0, 1, 2))
    g = (g - g.mean()) / g.std()
    rho = np.exp(g - 0.5)
    return rho / rho.mean()


@dataclasses.dataclass
class Halos:
    pos: np.ndarray      # [n, 3] Mpc/h
    vel: np.ndarray      # [n, 3] km/s
    mass: np.ndarray     # [n] Msun/h
    radius: np.ndarray   # [n] Mpc/h


def make_halos(box_L: float, n_gal_target: int, seed: int,
               hod=HOD_Z09) -> Halos:
    rng = np.random.default_rng(seed)
    ng = 64
    rho = _lognormal_field(rng, ng)
    n_halo_mean = n_gal_target / _mean_gal_per_halo(hod)
    counts = rng.poisson(n_halo_mean * rho.reshape(-1) / rho.size)
    cells = np.repeat(np.arange(rho.size), counts)
    n = cells.size
    cz = cells % ng
    cy = (cells // ng) % ng
    cx = cells // (ng * ng)
    cell_L = box_L / ng
    pos = (np.stack([cx, cy, cz], axis=1) + rng.random((n, 3))) * cell_L
    lnm, _, _, cdf = _mass_grid()
    mass = np.exp(np.interp(rng.random(n), cdf, lnm))
    vel = rng.normal(0.0, 300.0, size=(n, 3))
    radius = 1.6 * (mass / 1e15) ** (1.0 / 3.0)
    return Halos(pos % box_L, vel, mass, radius)


def _uniform_in_sphere(rng, n):
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = rng.random(n) ** (1.0 / 3.0)
    return d * r[:, None]


@dataclasses.dataclass
class Catalogue:
    pos: np.ndarray            # [n, 3] float64, in [0, L)
    vel: np.ndarray            # [n, 3] float32, km/s
    halo_id: np.ndarray        # [n] int64
    is_central: np.ndarray     # [n] bool
    box_L: float

    @property
    def n(self) -> int:
        return self.pos.shape[0]


def make_catalogue(w: Workload, seed: int = 0, hod=HOD_Z09) -> Catalogue:
    """Draw a galaxy catalogue for workload ``w`` (positions not RSD-shifted)."""
    return make_catalogue_box(w.box_L, w.n_gal, seed, hod)


def make_catalogue_box(box_L: float, n_gal: int, seed: int,
                       hod=HOD_Z09) -> Catalogue:
    halos = make_halos(box_L, n_gal, seed, hod)
    rng = np.random.default_rng([seed, 1])
    ncen, nsat = hod_mean_occupation(halos.mass, hod)
    has_cen = rng.random(halos.mass.size) < ncen
    n_sat = rng.poisson(nsat)
    cen_idx = np.nonzero(has_cen)[0]
    sat_idx = np.repeat(np.arange(halos.mass.size), n_sat)
    off = _uniform_in_sphere(rng, sat_idx.size) * halos.radius[sat_idx, None]
    sigma_v = np.sqrt(G_NEWTON * halos.mass / (2.0 * halos.radius))
    sat_vel = halos.vel[sat_idx] + rng.standard_normal((sat_idx.size, 3)) * sigma_v[sat_idx, None]
    pos = np.concatenate([halos.pos[cen_idx], halos.pos[sat_idx] + off])
    vel = np.concatenate([halos.vel[cen_idx], sat_vel])
    hid = np.concatenate([cen_idx, sat_idx]).astype(np.int64)
    isc = np.concatenate([np.ones(cen_idx.size, bool), np.zeros(sat_idx.size, bool)])
    pos = np.mod(pos, box_L)
    pos[pos >= box_L] = 0.0
    return Catalogue(pos.astype(np.float64), vel.astype(np.float32), hid, isc, box_L)


def make_uniform(box_L: float, n: int, seed: int) -> np.ndarray:
    """Poisson (uniform) positions in the box, [n, 3] float64."""
    rng = np.random.default_rng([seed, 7])
    return rng.random((n, 3)) * box_L


def make_weights(n: int, seed: int, lo: float = 0.25, hi: float = 1.0) -> np.ndarray:
    """Positive per-galaxy weights, [n] float32."""
    rng = np.random.default_rng([seed, 11])
    return (lo + (hi - lo) * rng.random(n)).astype(np.float32)


def subsample(cat: Catalogue, n_max: Optional[int], seed: int = 0) -> Catalogue:
    if n_max is None or cat.n <= n_max:
        return cat
    rng = np.random.default_rng([seed, 3])
    idx = np.sort(rng.choice(cat.n, n_max, replace=False))
    return Catalogue(cat.pos[idx], cat.vel[idx], cat.halo_id[idx],
                     cat.is_central[idx], cat.box_L)


@dataclasses.dataclass
class Candidates:
    """Candidate galaxies whose weights are soft HOD occupations: one central
    candidate per halo and K satellite candidates per halo that can host
    satellites, at positions drawn once from the seed (so that a change of
    HOD parameters changes only the weights)."""
    pos: np.ndarray      # [n, 3] float64
    vel: np.ndarray      # [n, 3] float32
    mass: np.ndarray     # [n] float64, host halo mass
    kind: np.ndarray     # [n] int32, 0 central, 1 satellite
    kh: np.ndarray       # [n] float32, satellite candidates of the halo (1 for centrals)
    box_L: float

    @property
    def n(self) -> int:
        return self.pos.shape[0]


def make_candidates(box_L: float, n_gal: int, seed: int, hod=HOD_Z09,
                    min_ncen: float = 1e-3) -> Candidates:
    halos = make_halos(box_L, n_gal, seed, hod)
    rng = np.random.default_rng([seed, 5])
    ncen, nsat = hod_mean_occupation(halos.mass, hod)
    log_mcut, _, _, _, kappa = hod
    cen = np.nonzero(ncen > min_ncen)[0]
    # halos above 10^-0.2 kappa M_cut may host satellites under nearby HODs
    can_sat = halos.mass > 10.0 ** (log_mcut - 0.2) * kappa * 0.999
    k = np.where(can_sat, np.maximum(1, np.ceil(2.0 * nsat)), 0).astype(np.int64)
    sat = np.repeat(np.arange(halos.mass.size), k)
    off = _uniform_in_sphere(rng, sat.size) * halos.radius[sat, None]
    sigma_v = np.sqrt(G_NEWTON * halos.mass / (2.0 * halos.radius))
    sat_vel = halos.vel[sat] + rng.standard_normal((sat.size, 3)) * sigma_v[sat, None]
    pos = np.mod(np.concatenate([halos.pos[cen], halos.pos[sat] + off]), box_L)
    pos[pos >= box_L] = 0.0
    vel = np.concatenate([halos.vel[cen], sat_vel]).astype(np.float32)
    mass = np.concatenate([halos.mass[cen], halos.mass[sat]])
    kind = np.concatenate([np.zeros(cen.size, np.int32), np.ones(sat.size, np.int32)])
    kh = np.concatenate([np.ones(cen.size), k[sat]]).astype(np.float32)
    return Candidates(pos, vel, mass, kind, kh, box_L)


def many_mocks(n_mocks: int = 64, seed0: int = 0):
    """The uneven many-mock batch: for mock s, box L ~ U[256, 1100] Mpc/h, mesh
    N = the power of two nearest L (cells of about 1 Mpc/h) clipped to
    [256, 1024], target galaxy count log-uniform on [2e4, 4e5], HOD
    parameters within +-0.2 dex of HOD_Z09 (added to the two log-masses,
    a factor 10^U(-0.2, 0.2) on sigma, alpha and kappa); the paper-scale
    binning (20 x 5 pair bins on s < 10, 10 x 5 correlation bins on
    10 < r < 60), CIC, real space. Returns [(Workload, hod)], one per mock
    (draw its catalogue with make_catalogue(w, seed, hod))."""
    out = []
    for s in range(seed0, seed0 + n_mocks):
        rng = np.random.default_rng([s, 55])
        L = float(rng.uniform(256.0, 1100.0))
        N = int(2 ** int(np.clip(np.round(np.log2(L)), 8, 10)))
        n_gal = int(round(math.exp(rng.uniform(math.log(2e4), math.log(4e5)))))
        d = rng.uniform(-0.2, 0.2, 5)
        t = HOD_Z09
        hod = (t[0] + d[0], t[1] + d[1], t[2] * 10 ** d[2], t[3] * 10 ** d[3], t[4] * 10 ** d[4])
        w = Workload(f"mock_{s}", L, N, 1, n_gal, _edges(0, 10, 20), 5, _edges(10, 60, 10), 5,
                     False, 0)
        out.append((w, hod))
    return out
