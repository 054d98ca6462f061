"""Seeded synthetic cell inputs for the thermochemical step.

This module only draws inputs: it holds none of the method's arithmetic and is
shared by the CUDA path's tests/benchmark and by the oracle's tests.  Every
array is float64, structure-of-arrays, one entry per cell, CGS units.

Recipes (stand-ins for the paper's Bonnor-Ebert, HII-region and GMC runs,
which are full simulations this library does not reproduce):

* ``cells_uniform``  -- independent draws (4096 cells = one 16^3 block):
  log10 n_H ~ U(0, 6); log10 T_g ~ U(1, 4); T_d ~ U(8, 30);
  log10 y_H+ ~ U(-8, -1) with y_e = y_H+ (charge neutrality);
  y_H2 = U(0, 1) * (1 - y_e) / 2 (so y_H = 1 - 2 y_H2 - y_e >= 0);
  log10 G0 ~ U(-2, 4); log10 n_EUV ~ U(-6, 2); log10 N_H2 ~ U(14, 22);
  E_IR = (c / c~) a T_d^4 (IR radiation in equilibrium with the dust).
* ``cells_grf``      -- the same marginals on an n^3 periodic grid, each field
  an independent Gaussian random field (white noise convolved with a
  Gaussian of sigma = 8 cells, standardised) mapped through the normal CDF
  and the marginal's inverse CDF (a Gaussian copula).
* ``cells_amr``      -- 3000 blocks of 8^3 cells on levels 0..6 nested around a
  collapsing core: n_H = clamp(1e8 (r / r_c)^-2, 1e2, 1e8) with r_c the finest
  cell size; a central EUV/FUV source diluted as 1/r^2 and extinguished by the
  analytic column of that profile; T_g = 10 + (1e4 - 10) exp(-tau_EUV);
  per-level time step dt_l = 1e3 yr / 2^l.
* ``cells_gmc``      -- an n^3 GMC-like grid: ln n_H Gaussian (mean n 100 cm^-3,
  sigma_ln 1.5) through one Gaussian random field, log10 T_g linearly
  anti-correlated with it and clamped to 10..1e4 K, 8 seeded point sources
  whose EUV/FUV fields fall as 1/r^2 and are shielded by a local column
  n_H min(r, 8 dx); dt = 1e3 yr, dust-capacity factor 100.
* ``cells_be``       -- the initial Bonnor-Ebert sphere of the collapse tests
  (Sec. 4.3): a critical isothermal sphere (dimensionless radius 6.45, the
  Lane-Emden profile integrated here), density raised by 1.2, central
  n_H = 1.2e4 cm^-3, the edge density outside; nested grids with l_max = 2,
  each level 8^3 blocks of 8^3 cells, the level-0 box spanning the sphere's
  diameter and each finer level the inner half of the one above (1408 leaf
  blocks, 720,896 cells); T_g and abundances are the paper's one-zone values
  for the metallicity (Table BEsphere: y_H2 and y_H+ as printed, y_e = y_H+,
  y_H from H-nuclei conservation, which matches the printed y_H to its
  rounding), T_d = T_g, no UV (G0 = n_EUV = 0: the test evolves IR radiation
  only), E_IR = (c / c~) a T_d^4, N_H2 = y_H2 n_H r; synchronous dt = half the
  finest level's sound-crossing time of a cell (5.2e3 yr, the same for every
  metallicity because the sphere scales with the sound speed).
"""
from __future__ import annotations

import numpy as np

YR = 3.15576e7          # s
PC = 3.0857e18          # cm
_A_RAD = 7.565733250e-15
_C_OVER_CRED = 1.0e4    # c / c~ for the reduced light speed c~ = 1e-4 c

FIELDS = ("n_H", "T_g", "T_d", "E_IR", "y_H2", "y_e", "G0", "n_EUV", "N_H2")


def _e_ir(T_d):
    return _C_OVER_CRED * _A_RAD * T_d ** 4


def _finish(c: dict) -> dict:
    for k in FIELDS:
        c[k] = np.ascontiguousarray(c[k], dtype=np.float64).reshape(-1)
    return c


def cells_uniform(n: int = 4096, seed: int = 1001) -> dict:
    """Independently drawn cells (see the module docstring)."""
    rng = np.random.default_rng(seed)
    u = rng.random((9, n))
    c = {}
    c["n_H"] = 10.0 ** (6.0 * u[0])
    c["T_g"] = 10.0 ** (1.0 + 3.0 * u[1])
    c["T_d"] = 8.0 + 22.0 * u[2]
    c["y_e"] = 10.0 ** (-8.0 + 7.0 * u[3])
    c["y_H2"] = u[4] * (1.0 - c["y_e"]) / 2.0
    c["G0"] = 10.0 ** (-2.0 + 6.0 * u[5])
    c["n_EUV"] = 10.0 ** (-6.0 + 8.0 * u[6])
    c["N_H2"] = 10.0 ** (14.0 + 8.0 * u[7])
    c["E_IR"] = _e_ir(c["T_d"])
    return _finish(c)


def _grf_uniform(rng, n: int, sigma: float = 8.0) -> np.ndarray:
    """U(0,1) field with the spatial correlation of a Gaussian-smoothed GRF."""
    from scipy.special import ndtr
    w = rng.standard_normal((n, n, n))
    k = np.fft.fftfreq(n)
    kr = np.fft.rfftfreq(n)
    k2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + kr[None, None, :] ** 2
    filt = np.exp(-2.0 * (np.pi * sigma) ** 2 * k2)   # FT of a unit-sum Gaussian, periodic
    g = np.fft.irfftn(np.fft.rfftn(w) * filt, s=(n, n, n), axes=(0, 1, 2))
    g = (g - g.mean()) / g.std()
    return ndtr(g)


def _grf_normal(rng, n: int, sigma: float = 8.0) -> np.ndarray:
    w = rng.standard_normal((n, n, n))
    k = np.fft.fftfreq(n)
    kr = np.fft.rfftfreq(n)
    k2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + kr[None, None, :] ** 2
    filt = np.exp(-2.0 * (np.pi * sigma) ** 2 * k2)
    g = np.fft.irfftn(np.fft.rfftn(w) * filt, s=(n, n, n), axes=(0, 1, 2))
    return (g - g.mean()) / g.std()


def cells_grf(n: int = 128, seed: int = 1002) -> dict:
    """n^3 grid, cell-uniform marginals through Gaussian-copula random fields."""
    rng = np.random.default_rng(seed)
    u = [_grf_uniform(rng, n) for _ in range(8)]
    c = {}
    c["n_H"] = 10.0 ** (6.0 * u[0])
    c["T_g"] = 10.0 ** (1.0 + 3.0 * u[1])
    c["T_d"] = 8.0 + 22.0 * u[2]
    c["y_e"] = 10.0 ** (-8.0 + 7.0 * u[3])
    c["y_H2"] = u[4] * (1.0 - c["y_e"]) / 2.0
    c["G0"] = 10.0 ** (-2.0 + 6.0 * u[5])
    c["n_EUV"] = 10.0 ** (-6.0 + 8.0 * u[6])
    c["N_H2"] = 10.0 ** (14.0 + 8.0 * u[7])
    c["E_IR"] = _e_ir(c["T_d"])
    return _finish(c)


def _morton3(ix, iy, iz):
    def spread(v):
        v = v.astype(np.uint64)
        out = np.zeros_like(v)
        for b in range(10):
            out |= ((v >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b)
        return out
    return spread(ix) | (spread(iy) << np.uint64(1)) | (spread(iz) << np.uint64(2))


AMR_LEVEL_COUNTS = (512, 512, 512, 488, 400, 320, 256)   # sums to 3000


def cells_amr(seed: int = 1004, L0_pc: float = 1.0):
    """3000 blocks of 8^3 cells over levels 0..6 (see the module docstring).

    Returns (cells, block_offset[int64, n_blocks+1], block_dt[float64],
    block_level[int32])."""
    rng = np.random.default_rng(seed)
    L0 = L0_pc * PC
    nb = 8                        # blocks per edge of each level's nest
    bc = 8                        # cells per block edge
    r_c = L0 / (nb * bc * 2 ** 6)  # finest cell size
    centre = np.full(3, 0.5 * L0)
    blocks = []                   # (level, origin[3], edge)
    for lev, count in enumerate(AMR_LEVEL_COUNTS):
        edge = L0 / nb / 2 ** lev
        lo = centre - 0.5 * nb * edge
        ii = np.arange(nb)
        ix, iy, iz = np.meshgrid(ii, ii, ii, indexing="ij")
        ix, iy, iz = ix.ravel(), iy.ravel(), iz.ravel()
        org = lo[None, :] + edge * np.stack([ix, iy, iz], 1)
        rad = np.linalg.norm(org + 0.5 * edge - centre[None, :], axis=1)
        order = np.lexsort((_morton3(ix, iy, iz), np.round(rad / edge, 9)))
        for j in order[:count]:
            blocks.append((lev, org[j], edge))
    nblk = len(blocks)
    ncell = nblk * bc ** 3
    pos = np.empty((ncell, 3))
    lvl = np.empty(nblk, np.int32)
    g = (np.arange(bc) + 0.5) / bc
    gx, gy, gz = np.meshgrid(g, g, g, indexing="ij")
    local = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], 1)  # x-fastest order is immaterial
    for b, (lev, org, edge) in enumerate(blocks):
        pos[b * bc ** 3:(b + 1) * bc ** 3] = org[None, :] + edge * local
        lvl[b] = lev
    r = np.maximum(np.linalg.norm(pos - centre[None, :], axis=1), 0.5 * r_c)
    n = np.clip(1e8 * (r / r_c) ** -2, 1e2, 1e8)
    # column from the centre: n = 1e8 inside r_c, 1e8 (r/r_c)^-2 out to r_100 = 1e3 r_c, 1e2 beyond
    r100 = 1e3 * r_c
    NH = np.where(r <= r_c, 1e8 * r,
                  np.where(r <= r100, 1e8 * r_c + 1e8 * r_c ** 2 * (1.0 / r_c - 1.0 / r),
                           1e8 * r_c + 1e8 * r_c ** 2 * (1.0 / r_c - 1.0 / r100) + 1e2 * (r - r100)))
    N_S = 1e8 * r_c + 1e8 * r_c ** 2 * (1.0 / r_c - 1.0 / (32.0 * r_c))  # tau_EUV = 1 at 32 r_c
    tau_euv = NH / N_S
    tau_fuv = 1e-21 * NH
    r0 = 32.0 * r_c
    c = {}
    c["n_H"] = n
    c["T_g"] = 10.0 + (1e4 - 10.0) * np.exp(-tau_euv)
    c["G0"] = 1e4 * (r0 / r) ** 2 * np.exp(-tau_fuv)
    c["n_EUV"] = 1e2 * (r0 / r) ** 2 * np.exp(-tau_euv)
    u = rng.random((3, ncell))
    c["T_d"] = 8.0 + 22.0 * u[0]
    c["y_e"] = 10.0 ** (-8.0 + 7.0 * u[1])
    c["y_H2"] = u[2] * (1.0 - c["y_e"]) / 2.0
    c["N_H2"] = np.maximum(c["y_H2"] * n * r, 0.0)
    c["E_IR"] = _e_ir(c["T_d"])
    block_offset = np.arange(nblk + 1, dtype=np.int64) * bc ** 3
    block_dt = 1e3 * YR / 2.0 ** lvl.astype(np.float64)
    return _finish(c), block_offset, block_dt, lvl


def cells_gmc(n: int = 256, seed: int = 1005, box_pc: float = 3.0) -> dict:
    """n^3 GMC-like grid with 8 point sources (see the module docstring)."""
    rng = np.random.default_rng(seed)
    dx = box_pc * PC / n
    z = _grf_normal(rng, n)
    mu_ln = np.log(100.0) - 0.5 * 1.5 ** 2
    c = {}
    nH = np.exp(mu_ln + 1.5 * z)
    c["n_H"] = nH
    c["T_g"] = 10.0 ** np.clip(2.5 - 1.5 * z / 2.0, 1.0, 4.0)
    uTd, uye, uy2 = (_grf_uniform(rng, n) for _ in range(3))
    c["T_d"] = 8.0 + 22.0 * uTd
    c["y_e"] = 10.0 ** (-8.0 + 7.0 * uye)
    c["y_H2"] = uy2 * (1.0 - c["y_e"]) / 2.0
    src = rng.random((8, 3)) * n
    S_fuv = 10.0 ** rng.uniform(2.0, 5.0, 8)     # G0 one cell away
    S_euv = 10.0 ** rng.uniform(0.0, 3.0, 8)     # n_EUV [cm^-3] one cell away
    ii = np.arange(n) + 0.5
    G0 = np.zeros((n, n, n))
    nE = np.zeros((n, n, n))
    for s in range(8):
        d2 = ((ii[:, None, None] - src[s, 0]) ** 2 + (ii[None, :, None] - src[s, 1]) ** 2 +
              (ii[None, None, :] - src[s, 2]) ** 2)
        rc = np.sqrt(np.maximum(d2, 0.25))
        Ncol = nH * np.minimum(rc, 8.0) * dx
        G0 += S_fuv[s] / rc ** 2 * np.exp(-1e-21 * Ncol)
        nE += S_euv[s] / rc ** 2 * np.exp(-6.3e-18 * Ncol)
    c["G0"] = G0
    c["n_EUV"] = nE
    c["N_H2"] = c["y_H2"] * nH * 8.0 * dx
    c["E_IR"] = _e_ir(c["T_d"])
    return _finish(c)


# Table BEsphere: initial T_g [K], y_H2 and y_H+ of the Bonnor-Ebert spheres
# by metallicity Z / Z_sun (Sec. 4.3).
BE_SEEDS = {1.0: (5.0, 4.98e-1, 1.27e-7), 1e-2: (21.0, 3.47e-2, 1.99e-7), 1e-4: (190.0, 1.18e-3, 8.29e-7)}


def _lane_emden(xi_max: float = 6.45, h: float = 1e-3):
    """Isothermal Lane-Emden solution psi(xi) (rho = rho_c exp(-psi)), RK4."""
    def f(x, y):
        psi, dpsi = y
        return np.array([dpsi, np.exp(-psi) - 2.0 * dpsi / x])
    x = 1e-4
    y = np.array([x * x / 6.0, x / 3.0])     # series start
    xs, ps = [0.0, x], [0.0, y[0]]
    while x < xi_max:
        k1 = f(x, y)
        k2 = f(x + h / 2, y + h / 2 * k1)
        k3 = f(x + h / 2, y + h / 2 * k2)
        k4 = f(x + h, y + h * k3)
        y = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        x += h
        xs.append(x)
        ps.append(y[0])
    return np.array(xs), np.array(ps)


def cells_be(Z: float = 1.0, levels: int = 3):
    """Initial Bonnor-Ebert sphere on nested grids (see the module docstring).
    Returns (cells, block_offset, block_level), blocks of 8^3 cells stored
    contiguously (x fastest inside a block)."""
    T0, y2, yp = BE_SEEDS[Z]
    b = np.arange(8)
    bz, by, bx = (a.reshape(-1) for a in np.meshgrid(b, b, b, indexing="ij"))
    inner = (bz >= 2) & (bz <= 5) & (by >= 2) & (by <= 5) & (bx >= 2) & (bx <= 5)
    c8 = np.arange(8)
    cz, cy, cx = (a.reshape(-1) for a in np.meshgrid(c8, c8, c8, indexing="ij"))
    xi_max = 6.45
    xs, ps = _lane_emden(xi_max)
    r_list, lev = [], []
    for l in range(levels):
        keep = np.ones(512, bool) if l == levels - 1 else ~inner
        h = xi_max / 32.0 / 2.0 ** l       # cell size in units of the BE length
        for k in np.nonzero(keep)[0]:
            x = (bx[k] * 8 + cx - 32 + 0.5) * h
            y = (by[k] * 8 + cy - 32 + 0.5) * h
            z = (bz[k] * 8 + cz - 32 + 0.5) * h
            r_list.append(np.sqrt(x * x + y * y + z * z))
            lev.append(l)
    xi = np.concatenate(r_list)
    psi = np.interp(np.minimum(xi, xi_max), xs, ps)
    nH = 1.2e4 * np.exp(-psi)
    # BE length c_s / sqrt(4 pi G rho_c) in cm (isothermal c_s, mu = 2.3)
    kB, mH, G = 1.380649e-16, 1.6726e-24, 6.674e-8
    cs = np.sqrt(kB * T0 / (2.3 * mH))
    Lbe = cs / np.sqrt(4.0 * np.pi * G * 1.4 * mH * 1.2e4)
    n = len(xi)
    c = {}
    c["n_H"] = nH
    c["T_g"] = np.full(n, T0)
    c["T_d"] = np.full(n, T0)
    c["y_e"] = np.full(n, yp)
    c["y_H2"] = np.full(n, y2)
    c["G0"] = np.zeros(n)
    c["n_EUV"] = np.zeros(n)
    c["N_H2"] = y2 * nH * np.maximum(xi, 0.5 * xi_max / 32.0 / 2.0 ** (levels - 1)) * Lbe
    c["E_IR"] = _e_ir(c["T_d"])
    block_offset = np.arange(len(lev) + 1, dtype=np.int64) * 512
    return _finish(c), block_offset, np.asarray(lev, dtype=np.int32)


def be_dt(levels: int = 3) -> float:
    """Synchronous step of the sphere: half the finest cell's sound-crossing
    time (independent of T_g, see the module docstring)."""
    kB, mH, G = 1.380649e-16, 1.6726e-24, 6.674e-8
    # dx_f / c_s = (6.45 / 32 / 2^(levels-1)) / sqrt(4 pi G rho_c)
    return 0.5 * (6.45 / 32.0 / 2.0 ** (levels - 1)) / np.sqrt(4.0 * np.pi * G * 1.4 * mH * 1.2e4)


def cells_extreme(n: int = 4096, seed: int = 2024) -> dict:
    """Independent cells over ranges wider than any workload's, for
    robustness tests: log n_H ~ U(-2, 12); log T_g ~ U(log 3, 5);
    log T_d ~ U(log 3, log 3 + 3); y_e within 1e-8 of 1 for a fifth of the
    cells, else log y_e ~ U(-10, 0); y_H2 within a factor 1 - 1e-8 of
    (1 - y_e)/2 for 30 % of the cells, else U(0, 1) (1 - y_e)/2;
    log G0 ~ U(-3, 6); log n_EUV ~ U(-8, 4); log N_H2 ~ U(12, 25);
    E_IR = (c / c~) a T_d^4."""
    rng = np.random.default_rng(seed)
    u = rng.random((10, n))
    c = {}
    c["n_H"] = 10.0 ** (-2.0 + 14.0 * u[0])
    c["T_g"] = 10.0 ** (np.log10(3.0) + (5.0 - np.log10(3.0)) * u[1])
    c["T_d"] = 10.0 ** (np.log10(3.0) + 3.0 * u[2])
    ye = np.where(u[3] < 0.2, 1.0 - 10.0 ** (-8.0 * u[4]), 10.0 ** (-10.0 + 10.0 * u[4]))
    c["y_e"] = np.minimum(ye, 1.0)
    half = (1.0 - c["y_e"]) / 2.0
    c["y_H2"] = np.where(u[5] < 0.3, half * (1.0 - 10.0 ** (-8.0 * u[6])), u[6] * half)
    c["G0"] = 10.0 ** (-3.0 + 9.0 * u[7])
    c["n_EUV"] = 10.0 ** (-8.0 + 12.0 * u[8])
    c["N_H2"] = 10.0 ** (12.0 + 13.0 * u[9])
    c["E_IR"] = _e_ir(c["T_d"])
    return _finish(c)


def paper_case(case: int) -> dict:
    """One cell of the paper's chemistry tests (Sec. 3.5, Table chemistryTest)."""
    if case == 1:
        c = dict(n_H=1e5, T_g=10.0, T_d=10.0, y_H2=1e-5, y_e=1e-5)
    elif case == 2:
        c = dict(n_H=1e2, T_g=12000.0, T_d=75.0, y_H2=1e-5, y_e=1e-5)
    else:
        raise ValueError(case)
    c.update(G0=0.0, n_EUV=0.0, N_H2=0.0, E_IR=_e_ir(c["T_d"]))
    return _finish({k: np.array([v]) for k, v in c.items()})


def subset(cells: dict, idx) -> dict:
    return {k: np.ascontiguousarray(v[idx]) for k, v in cells.items()}


def concat(*parts: dict) -> dict:
    return {k: np.concatenate([p[k] for p in parts]) for k in FIELDS}


def block_major(cells: dict, n: int, b: int = 16):
    """Reorder an n^3 x-fastest grid into contiguous b^3 blocks (the layout of
    a block-structured AMR code).  Returns (cells, block_offset)."""
    assert n % b == 0
    nb = n // b
    out = {}
    for k, v in cells.items():
        a = np.asarray(v).reshape(nb, b, nb, b, nb, b)          # (z, z', y, y', x, x')
        out[k] = np.ascontiguousarray(a.transpose(0, 2, 4, 1, 3, 5)).reshape(-1)
    block_offset = np.arange(nb ** 3 + 1, dtype=np.int64) * b ** 3
    return out, block_offset
