"""Seeded synthetic inputs for the TTI and elastic propagators.

This module is shared by the FP64 oracle (``oracle/``), the GPU library's
tests and ``bench.py``.  It holds no arithmetic of the propagators: it only
draws seeded random fields, shapes them into velocity / anisotropy / density
models with the scales of the paper's experiments (Sec. III-B: 12.5 m grid,
40-cell absorbing layer; Sec. IV-C: space order 12 elastic), samples the
source wavelet and lays out sources and receivers.

Units: velocities in km/s, density in g/cc, angles in radians, coordinates in
metres with the origin at the first PHYSICAL grid point and z pointing down.
Every array is float32, C-contiguous, indexed ``[x][y][z]`` on the physical
grid.  The absorbing layer is added by the propagators themselves.

Random numbers come from ``numpy.random.Generator(PCG64(seed))``, which
draws the same stream on every platform.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TTI = 1
ELASTIC = 2
ACOUSTIC = 3
ELASTIC2D = 4      # x-z plane, ny = 1

DEG = math.pi / 180.0


# --------------------------------------------------------------------------
# primitive generators
# --------------------------------------------------------------------------
def ricker(f0: float, dt: float, nt: int, t0: float | None = None) -> np.ndarray:
    """Ricker wavelet of peak frequency ``f0`` [Hz] sampled at t = n*dt.

    q(t) = (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2), t0 = 1/f0.
    """
    if t0 is None:
        t0 = 1.0 / f0
    t = np.arange(nt, dtype=np.float64) * dt - t0
    a = (math.pi * f0 * t) ** 2
    return ((1.0 - 2.0 * a) * np.exp(-a)).astype(np.float32)


def _gauss_axis(a: np.ndarray, sigma: float, axis: int) -> np.ndarray:
    """Periodic Gaussian smoothing of ``a`` along one axis (FFT)."""
    n = a.shape[axis]
    if sigma <= 0 or n < 2:
        return a
    f = np.fft.rfftfreq(n)
    tf = np.exp(-0.5 * (2.0 * math.pi * f * sigma) ** 2)
    shape = [1] * a.ndim
    shape[axis] = tf.size
    A = np.fft.rfft(a, axis=axis)
    A *= tf.reshape(shape)
    return np.fft.irfft(A, n=n, axis=axis)


def smooth_noise(shape, sigma_cells, seed: int) -> np.ndarray:
    """Gaussian-filtered white noise rescaled to [0, 1] (float64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.standard_normal(size=tuple(shape))
    if np.isscalar(sigma_cells):
        sigma_cells = (sigma_cells,) * len(shape)
    for ax, s in enumerate(sigma_cells):
        a = _gauss_axis(a, float(s), ax)
    lo, hi = a.min(), a.max()
    if hi <= lo:
        return np.zeros(shape)
    return (a - lo) / (hi - lo)


def rescale(u01: np.ndarray, lo: float, hi: float) -> np.ndarray:
    return lo + (hi - lo) * u01


def line_receivers(x0, dx, n, y, z) -> np.ndarray:
    r = np.zeros((n, 3), np.float32)
    r[:, 0] = x0 + dx * np.arange(n)
    r[:, 1] = y
    r[:, 2] = z
    return r


def carpet_receivers(x0, y0, dx, nx, ny, z) -> np.ndarray:
    xs = x0 + dx * np.arange(nx)
    ys = y0 + dx * np.arange(ny)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    r = np.zeros((nx * ny, 3), np.float32)
    r[:, 0] = X.ravel()
    r[:, 1] = Y.ravel()
    r[:, 2] = z
    return r


def cfl_dt(h: float, vmax_kms: float, cfl: float = 0.4) -> float:
    """Time step of a configuration: dt = cfl * h / vmax (vmax in km/s)."""
    return float(np.float32(cfl * h / (vmax_kms * 1000.0)))


# --------------------------------------------------------------------------
# problem container
# --------------------------------------------------------------------------
@dataclass
class Problem:
    kind: int
    nx: int
    ny: int
    nz: int
    nbl: int
    h: float
    so: int
    nt: int
    dt: float
    model: dict            # TTI: vp, eps, delta, theta, phi ; ELASTIC: vp, vs, rho ; ACOUSTIC: vp
    src: np.ndarray        # [nsrc, 3] float32
    wavelet: np.ndarray    # [nsrc, nt] float32
    rec: np.ndarray        # [nrec, 3] float32
    name: str = ""
    extra: dict = field(default_factory=dict)
    vdamp: float = 0.0     # TTI damping reference velocity [m/s]; 0 = from model
    tti_op: int = 0        # TTI operator: 0 composed centred, 1 staggered pair (diagonal terms)

    @property
    def ncomp(self):
        return ((self.nx + 2 * self.nbl) * (self.ny + 2 * self.nbl)
                * (self.nz + 2 * self.nbl))

    def model_list(self):
        keys = {TTI: ("vp", "eps", "delta", "theta", "phi"), ELASTIC: ("vp", "vs", "rho"),
                ACOUSTIC: ("vp",), ELASTIC2D: ("vp", "vs", "rho")}[self.kind]
        return [np.ascontiguousarray(self.model[k], dtype=np.float32) for k in keys]


# --------------------------------------------------------------------------
# model recipes
# --------------------------------------------------------------------------
def two_layer_tti(nx, ny, nz, h, z_interface, top, bottom) -> dict:
    """Two-layer TTI model; ``top``/``bottom`` = (vp, eps, delta, theta, phi)."""
    zc = np.arange(nz) * h
    lower = (zc >= z_interface)[None, None, :]
    out = {}
    for i, k in enumerate(("vp", "eps", "delta", "theta", "phi")):
        a = np.where(lower, bottom[i], top[i]) * np.ones((nx, ny, 1))
        out[k] = np.ascontiguousarray(a, dtype=np.float32)
    return out


def layered_vp(nx, ny, nz, seed, nlayers=10, vmin=1.5, vmax=4.5, noise_sigma=16.0,
               noise_amp=0.25) -> np.ndarray:
    """``nlayers`` flat layers increasing from vmin to vmax [km/s] with depth,
    plus smooth noise, clipped to [vmin, vmax] (float64)."""
    z = np.arange(nz) / max(nz - 1, 1)
    layer = np.minimum((z * nlayers).astype(int), nlayers - 1)
    vlayer = vmin + (vmax - vmin) * layer / max(nlayers - 1, 1)
    noise = smooth_noise((nx, ny, nz), noise_sigma, seed) * 2.0 - 1.0
    return np.clip(vlayer[None, None, :] + noise_amp * (vmax - vmin) * noise, vmin, vmax)


def layered_tti(nx, ny, nz, seed, nlayers=10, vmin=1.5, vmax=4.5,
                noise_sigma=16.0, noise_amp=0.25, smooth_sigma=4.0,
                eps_max=0.3, theta_max_deg=40.0) -> dict:
    """Layered-plus-noise TTI model (recipe of the industry-scale TTI runs).

    vp: ``nlayers`` flat layers increasing from vmin to vmax with depth, plus
    smooth noise, clipped to [vmin, vmax].  Anisotropy follows the smoothed
    velocity (eps = eps_max*(vp_s-vmin)/(vmax-vmin), delta = eps/2, so that
    eps >= delta); tilt = dip of the smoothed-velocity iso-surfaces clipped
    to theta_max; azimuth = direction of the lateral gradient in [0, 90 deg].
    """
    vp = layered_vp(nx, ny, nz, seed, nlayers, vmin, vmax, noise_sigma, noise_amp)
    vs_ = vp.copy()
    for ax in range(3):
        vs_ = _gauss_axis(vs_, smooth_sigma, ax)
    eps = eps_max * np.clip((vs_ - vmin) / (vmax - vmin), 0.0, 1.0)
    delta = 0.5 * eps
    gx, gy, gz = np.gradient(vs_)
    gh = np.sqrt(gx * gx + gy * gy)
    theta = np.clip(np.arctan2(gh, np.abs(gz) + 1e-12), 0.0, theta_max_deg * DEG)
    phi = np.arctan2(np.abs(gy), np.abs(gx))
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return {"vp": f32(vp), "eps": f32(eps), "delta": f32(delta),
            "theta": f32(theta), "phi": f32(phi)}


def random_elastic(nx, ny, nz, seed, sigma_cells, vp_range=(1.5, 4.5),
                   rho_range=(1.0, 2.5), vp_vs=1.73) -> dict:
    """Smooth random isotropic elastic model (Gaussian-filtered noise)."""
    vp = rescale(smooth_noise((nx, ny, nz), sigma_cells, seed), *vp_range)
    rho = rescale(smooth_noise((nx, ny, nz), sigma_cells, seed + 1), *rho_range)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return {"vp": f32(vp), "vs": f32(vp / vp_vs), "rho": f32(rho)}


# --------------------------------------------------------------------------
# named workloads (seed = 20040 + index)
# --------------------------------------------------------------------------
def tti_two_layer(n=64, h=10.0, nbl=10, so=8, nt=150, f0=15.0, seed=20041,
                  nrec=64) -> Problem:
    """TTI forward, two-layer model, one Ricker source at depth 100 m.

    Default sizes: 64^3 physical at 10 m + 10-cell layer, space order 8,
    150 steps, 64 receivers on a line at 20 m depth.
    """
    z_if = (n // 2) * h
    top = (1.5, 0.0, 0.0, 0.0, 0.0)
    bot = (2.5, 0.2, 0.1, 30 * DEG, 45 * DEG)
    model = two_layer_tti(n, n, n, h, z_if, top, bot)
    dt = cfl_dt(h, 2.5 * math.sqrt(1.4))
    c = (n // 2) * h
    src = np.array([[c, c, min(100.0, (n - 1) * h)]], np.float32)
    wav = ricker(f0, dt, nt)[None, :]
    rec = line_receivers(0.0, (n - 1) * h / max(nrec - 1, 1), nrec, c, min(20.0, (n - 1) * h))
    return Problem(TTI, n, n, n, nbl, h, so, nt, dt, model, src, wav, rec,
                   name=f"tti-two-layer-{n}^3-so{so}-nt{nt}")


def elastic_random(n=256, h=10.0, nbl=20, so=8, nt=1000, f0=10.0, seed=20042,
                   corr_len=200.0, nrec_side=64, rec_dx=40.0) -> Problem:
    """Elastic forward/adjoint on a smooth random model, explosive source at the
    grid centre, a square carpet of receivers at the surface."""
    model = random_elastic(n, n, n, seed, corr_len / h)
    dt = cfl_dt(h, float(model["vp"].max()))
    c = (n // 2) * h
    src = np.array([[c, c, c]], np.float32)
    wav = ricker(f0, dt, nt)[None, :]
    ext = (n - 1) * h
    nside = min(nrec_side, int((ext - 20.0) // rec_dx) + 1) if ext > 20 else 1
    rec = carpet_receivers(min(20.0, ext), min(20.0, ext), rec_dx, nside, nside, 0.0)
    return Problem(ELASTIC, n, n, n, 0 + nbl, h, so, nt, dt, model, src, wav, rec,
                   name=f"elastic-random-{n}^3-so{so}-nt{nt}")


def tti_layered(nx=800, ny=800, nz=400, h=12.5, nbl=40, so=12, nt=3000, f0=12.0,
                seed=20043, rec_dx=40.0, rec_n=250, src_xy=None) -> Problem:
    """Industry-scale TTI forward on a layered-plus-noise model."""
    model = layered_tti(nx, ny, nz, seed)
    vmax = float(np.max(model["vp"] * np.sqrt(1 + 2 * model["eps"])))
    dt = cfl_dt(h, vmax)
    if src_xy is None:
        src_xy = ((nx // 2) * h * 1.0, (ny // 2) * h * 1.0)
    src = np.array([[src_xy[0], src_xy[1], 2 * h]], np.float32)
    wav = ricker(f0, dt, nt)[None, :]
    nrx = min(rec_n, int(((nx - 1) * h) // rec_dx) + 1)
    nry = min(rec_n, int(((ny - 1) * h) // rec_dx) + 1)
    rec = carpet_receivers(0.0, 0.0, rec_dx, nrx, nry, h)
    return Problem(TTI, nx, ny, nz, nbl, h, so, nt, dt, model, src, wav, rec,
                   name=f"tti-layered-{nx}x{ny}x{nz}-so{so}-nt{nt}")


def smooth_model(model: dict, sigma_cells: float, keys=("vp",)) -> dict:
    """Starting model for inversion: ``keys`` Gaussian-smoothed, the rest kept."""
    out = dict(model)
    for k in keys:
        a = model[k].astype(np.float64)
        for ax in range(3):
            a = _gauss_axis(a, sigma_cells, ax)
        out[k] = np.ascontiguousarray(a, dtype=np.float32)
    return out


def tti_gradient_problem(nx=400, ny=400, nz=300, h=12.5, nbl=40, so=12, nt=2000,
                         f0=12.0, seed=20044, rec_dx=25.0, rec_n=200,
                         smooth_m=150.0):
    """TTI FWI gradient workload: true model, smoothed starting model (vp only)."""
    true = tti_layered(nx, ny, nz, h, nbl, so, nt, f0, seed, rec_dx, rec_n)
    start = smooth_model(true.model, smooth_m / h)
    # keep the same dt for both models (the true model bounds vmax)
    p0 = Problem(TTI, nx, ny, nz, nbl, h, so, nt, true.dt, start, true.src,
                 true.wavelet, true.rec, name=true.name.replace("layered", "grad"))
    return true, p0


def perturbation(shape, nbl_free: int, seed: int, sigma_cells=3.0) -> np.ndarray:
    """Smooth seeded perturbation in [-1, 1], zero within ``nbl_free`` cells of
    the physical-grid faces (used by Taylor tests)."""
    d = smooth_noise(shape, sigma_cells, seed) * 2.0 - 1.0
    mask = np.zeros(shape)
    sl = tuple(slice(nbl_free, s - nbl_free) for s in shape)
    mask[sl] = 1.0
    return np.ascontiguousarray(d * mask, dtype=np.float32)


def random_state(n_fields, shape, seed, sigma_cells=1.5):
    """Seeded smooth random wavefield states (one-step parity tests)."""
    out = []
    for i in range(n_fields):
        u = smooth_noise(shape, sigma_cells, seed + i) * 2.0 - 1.0
        out.append(np.ascontiguousarray(u, dtype=np.float32))
    return out


# --------------------------------------------------------------------------
# batched shots on windows of one large model
# --------------------------------------------------------------------------
class UndulatingTTI:
    """A large layered TTI model given in closed form, so that any window of
    it can be drawn without building the whole volume.

    Layers of constant vp (``nlayers`` from vmin to vmax with depth) are
    bounded by interfaces that all follow one smooth seeded undulation
    U(x, y) (a sum of a few random 2D cosine modes with wavelengths of
    1.5-6 km and ``amp`` metres of total relief): a point (x, y, z) lies in
    layer floor((z - U(x, y)) / thickness).  Anisotropy follows the velocity
    (eps = eps_max (vp - vmin)/(vmax - vmin), delta = eps/2), the tilt is the
    dip of the interfaces (tan theta = |grad U|) and the azimuth that of
    grad U, folded to [0, 90 deg] -- the structure of the industry-scale
    TTI recipe, without its small-scale noise."""

    def __init__(self, seed, extent=(12500.0, 12500.0, 6250.0), nlayers=10, vmin=1.5,
                 vmax=4.5, amp=400.0, nmodes=6, eps_max=0.3):
        rng = np.random.default_rng(seed)
        self.extent, self.nlayers, self.vmin, self.vmax = extent, nlayers, vmin, vmax
        self.eps_max = eps_max
        lam = rng.uniform(1500.0, 6000.0, nmodes)
        ang = rng.uniform(0.0, 2 * math.pi, nmodes)
        self.k = np.stack([np.cos(ang), np.sin(ang)], 1) * (2 * math.pi / lam)[:, None]
        self.ph = rng.uniform(0.0, 2 * math.pi, nmodes)
        self.a = rng.uniform(0.5, 1.0, nmodes)
        self.a *= 0.5 * amp / self.a.sum()

    def window(self, ox, oy, nx, ny, nz, h) -> dict:
        """Model on the window whose first point is (ox, oy, 0) cells."""
        x = (ox + np.arange(nx)) * h
        y = (oy + np.arange(ny)) * h
        X, Y = np.meshgrid(x, y, indexing="ij")
        U = np.zeros((nx, ny))
        Ux = np.zeros((nx, ny))
        Uy = np.zeros((nx, ny))
        for (kx, ky), ph, a in zip(self.k, self.ph, self.a):
            arg = kx * X + ky * Y + ph
            U += a * np.cos(arg)
            s = -a * np.sin(arg)
            Ux += s * kx
            Uy += s * ky
        thick = self.extent[2] / self.nlayers
        vl = (self.vmin + (self.vmax - self.vmin) * np.arange(self.nlayers)
              / max(self.nlayers - 1, 1)).astype(np.float32)
        z = (np.arange(nz) * h).astype(np.float32)
        zeta = z[None, None, :] - U.astype(np.float32)[:, :, None] + np.float32(0.5 * thick)
        layer = np.clip(np.floor(zeta / np.float32(thick)), 0, self.nlayers - 1).astype(np.int8)
        vp = vl[layer]
        del zeta, layer
        eps = (np.float32(self.eps_max / (self.vmax - self.vmin)) * (vp - np.float32(self.vmin)))
        theta = np.arctan(np.hypot(Ux, Uy)).astype(np.float32)
        phi = np.arctan2(np.abs(Uy), np.abs(Ux)).astype(np.float32)
        full = lambda a2: np.ascontiguousarray(np.broadcast_to(a2[:, :, None], (nx, ny, nz)))
        return {"vp": vp, "eps": eps, "delta": np.ascontiguousarray(0.5 * eps, dtype=np.float32),
                "theta": full(theta), "phi": full(phi)}


def tti_batch_shots(nshots=8, nt=150, seed=20045, size_range=(200, 600), nz=300, h=12.5,
                    nbl=40, so=12, f0=12.0, global_cells=(1000, 1000, 500)):
    """Batched-gradient workload: ``nshots`` TTI shots on windows with
    nx, ny ~ U[size_range], nz fixed, at random offsets in a large
    undulating-layer model of ``global_cells`` cells at h; source at the
    window centre, 25 m deep; receivers every 4 cells at depth h.  Each shot
    is (true problem, starting problem): the starting model replaces vp by a
    linear increase with depth over the velocity range (other parameters
    true).  One dt (CFL of the global velocity range) for all shots."""
    rng = np.random.default_rng(seed)
    gx, gy, gz = global_cells
    model = UndulatingTTI(seed, extent=(gx * h, gy * h, gz * h))
    vmax = model.vmax * math.sqrt(1 + 2 * model.eps_max)
    dt = cfl_dt(h, vmax)
    shots = []
    for s in range(nshots):
        nx, ny = (int(v) for v in rng.integers(size_range[0], size_range[1] + 1, 2))
        ox = int(rng.integers(0, gx - nx + 1))
        oy = int(rng.integers(0, gy - ny + 1))
        m = model.window(ox, oy, nx, ny, nz, h)
        src = np.array([[(nx // 2) * h, (ny // 2) * h, 25.0]], np.float32)
        rec = carpet_receivers(0.0, 0.0, 4 * h, (nx - 1) // 4 + 1, (ny - 1) // 4 + 1, h)
        wav = ricker(f0, dt, nt)[None, :]
        name = f"tti-window-{nx}x{ny}x{nz}-at-{ox},{oy}-so{so}-nt{nt}"
        true = Problem(TTI, nx, ny, nz, nbl, h, so, nt, dt, m, src, wav, rec, name=name)
        z = (np.arange(nz) / max(nz - 1, 1)).astype(np.float32)
        v0 = model.vmin + (model.vmax - model.vmin) * z
        start = dict(m)
        start["vp"] = np.ascontiguousarray(np.broadcast_to(v0[None, None, :], (nx, ny, nz)),
                                           dtype=np.float32)
        p0 = Problem(TTI, nx, ny, nz, nbl, h, so, nt, dt, start, src, wav, rec,
                     name=name.replace("window", "window-start"))
        shots.append((true, p0))
    return shots


# --------------------------------------------------------------------------
# isotropic acoustic workloads
# --------------------------------------------------------------------------
def acoustic_layered(nx=800, ny=800, nz=400, h=12.5, nbl=40, so=12, nt=3000, f0=12.0,
                     seed=20046, rec_dx=40.0, rec_n=250) -> Problem:
    """Isotropic acoustic forward on the layered-plus-noise velocity of the
    industry-scale TTI recipe (same grid, order and geometry)."""
    vp = np.ascontiguousarray(layered_vp(nx, ny, nz, seed), dtype=np.float32)
    dt = cfl_dt(h, float(vp.max()))
    src = np.array([[(nx // 2) * h, (ny // 2) * h, 2 * h]], np.float32)
    wav = ricker(f0, dt, nt)[None, :]
    n = min(rec_n, int(((nx - 1) * h) // rec_dx) + 1)
    m = min(rec_n, int(((ny - 1) * h) // rec_dx) + 1)
    rec = carpet_receivers(0.0, 0.0, rec_dx, n, m, h)
    return Problem(ACOUSTIC, nx, ny, nz, nbl, h, so, nt, dt, {"vp": vp}, src, wav, rec,
                   name=f"acoustic-layered-{nx}x{ny}x{nz}-so{so}-nt{nt}")


def acoustic_small(shape=(37, 29, 45), nbl=7, h=10.0, so=8, nt=70, seed=3):
    """Small heterogeneous acoustic problem (parity tests): layered-plus-noise
    velocity, two sources, a carpet of receivers."""
    nx, ny, nz = shape
    vp = np.ascontiguousarray(layered_vp(nx, ny, nz, seed, noise_sigma=3.0), dtype=np.float32)
    dt = cfl_dt(h, float(vp.max()))
    src = np.array([[nx * h * 0.45 + 1.3, ny * h * 0.55 - 2.1, 3.3 * h],
                    [nx * h * 0.25, ny * h * 0.3 + 0.7, nz * h * 0.6]], np.float32)
    wav = np.vstack([ricker(25.0, dt, nt), 0.6 * ricker(18.0, dt, nt)]).astype(np.float32)
    rec = carpet_receivers(5.2, 7.1, 3.7 * h, 9, 7, 1.9 * h)
    return Problem(ACOUSTIC, nx, ny, nz, nbl, h, so, nt, dt, {"vp": vp}, src, wav, rec,
                   name=f"acoustic-small-{nx}x{ny}x{nz}-so{so}")


def acoustic_rtm_shots(nshots=8, nt=150, seed=20047, size_range=(200, 600), nz=300, h=12.5,
                       nbl=40, so=12, f0=12.0, global_cells=(1000, 1000, 500)):
    """RTM over many shots: ``nshots`` acoustic shots on windows with
    nx, ny ~ U[size_range], nz fixed, at random offsets in the undulating
    10-layer model (velocity only) of ``global_cells`` cells at h; source at
    the window centre, 25 m deep; receivers every 4 cells at depth h.  Each
    entry is (true problem, migration problem, (ox, oy, 0)): the migration
    velocity increases linearly with depth over the velocity range.  The
    stacked image is the sum of the shots' dJ/dm at their offsets in the
    global grid."""
    rng = np.random.default_rng(seed)
    gx, gy, gz = global_cells
    model = UndulatingTTI(seed, extent=(gx * h, gy * h, gz * h))
    dt = cfl_dt(h, model.vmax)
    shots = []
    for s in range(nshots):
        nx, ny = (int(v) for v in rng.integers(size_range[0], size_range[1] + 1, 2))
        ox = int(rng.integers(0, gx - nx + 1))
        oy = int(rng.integers(0, gy - ny + 1))
        vp = model.window(ox, oy, nx, ny, nz, h)["vp"]
        src = np.array([[(nx // 2) * h, (ny // 2) * h, 25.0]], np.float32)
        rec = carpet_receivers(0.0, 0.0, 4 * h, (nx - 1) // 4 + 1, (ny - 1) // 4 + 1, h)
        wav = ricker(f0, dt, nt)[None, :]
        name = f"acoustic-window-{nx}x{ny}x{nz}-at-{ox},{oy}-so{so}-nt{nt}"
        true = Problem(ACOUSTIC, nx, ny, nz, nbl, h, so, nt, dt, {"vp": vp}, src, wav, rec, name=name)
        z = (np.arange(nz) / max(nz - 1, 1)).astype(np.float32)
        v0 = model.vmin + (model.vmax - model.vmin) * z
        vmig = np.ascontiguousarray(np.broadcast_to(v0[None, None, :], (nx, ny, nz)), dtype=np.float32)
        p0 = Problem(ACOUSTIC, nx, ny, nz, nbl, h, so, nt, dt, {"vp": vmig}, src, wav, rec,
                     name=name.replace("window", "window-migration"))
        shots.append((true, p0, (ox, oy, 0)))
    return shots


# --------------------------------------------------------------------------
# 2D elastic workloads (x-z plane, ny = 1)
# --------------------------------------------------------------------------
def marine_elastic_2d(nx=1701, nz=701, h=5.0, nbl=40, so=8, nt=2000, f0=15.0, seed=20048,
                      water_depth=450.0, rec_dx=10.0) -> Problem:
    """2D elastic marine model standing in for the elastic Marmousi-II of the
    2D example: a water layer (vp 1.5 km/s, vs 0, rho 1.02 g/cc) over a
    layered elastic subsurface (vp 1.6 -> 4.5 km/s with depth plus smooth
    noise, vs = vp / 1.9, rho = 0.31 vp^0.25 (Gardner, vp in m/s));
    explosive source 10 m deep at the centre; pressure receivers every
    rec_dx at 5 m depth."""
    z = np.arange(nz) * h
    noise = smooth_noise((nx, 1, nz), 8.0, seed)[:, 0, :] * 2.0 - 1.0
    frac = np.clip((z - water_depth) / max(z[-1] - water_depth, h), 0.0, 1.0)
    vlayer = 1.6 + (4.5 - 1.6) * np.floor(frac * 12.0) / 11.0
    vp = np.clip(vlayer[None, :] + 0.25 * noise, 1.6, 4.5)
    water = (z < water_depth)[None, :]
    vp = np.where(water, 1.5, vp)
    vs = np.where(water, 0.0, vp / 1.9)
    rho = np.where(water, 1.02, 0.31 * (vp * 1000.0) ** 0.25)
    f32 = lambda a: np.ascontiguousarray(a[:, None, :], dtype=np.float32)
    model = {"vp": f32(vp), "vs": f32(vs), "rho": f32(rho)}
    dt = cfl_dt(h, float(vp.max()))
    src = np.array([[(nx // 2) * h, 0.0, 10.0]], np.float32)
    nrec = int(((nx - 1) * h) // rec_dx) + 1
    rec = np.zeros((nrec, 3), np.float32)
    rec[:, 0] = np.arange(nrec) * rec_dx
    rec[:, 2] = 5.0
    wav = ricker(f0, dt, nt)[None, :]
    return Problem(ELASTIC2D, nx, 1, nz, nbl, h, so, nt, dt, model, src, wav, rec,
                   name=f"elastic2d-marine-{nx}x{nz}-so{so}-nt{nt}")


def elastic2d_small(shape=(45, 38), nbl=7, h=10.0, so=8, nt=70, seed=4):
    """Small heterogeneous 2D elastic problem (parity tests): smooth random
    vp, vs, rho; two sources; a line of receivers."""
    nx, nz = shape
    m3 = random_elastic(nx, 1, nz, seed, 3.0)
    dt = cfl_dt(h, float(m3["vp"].max()))
    src = np.array([[nx * h * 0.45 + 1.3, 0.0, 3.3 * h], [nx * h * 0.25, 0.0, nz * h * 0.6]], np.float32)
    wav = np.vstack([ricker(25.0, dt, nt), 0.6 * ricker(18.0, dt, nt)]).astype(np.float32)
    rec = np.zeros((11, 3), np.float32)
    rec[:, 0] = 5.2 + (nx - 2) * h / 10.0 * np.arange(11)
    rec[:, 2] = 1.9 * h
    return Problem(ELASTIC2D, nx, 1, nz, nbl, h, so, nt, dt, m3, src, wav, rec,
                   name=f"elastic2d-small-{nx}x{nz}-so{so}")


def elastic_batch_shots(nshots=32, nt=1500, seed=20049, size_range=(200, 600), nz=300, h=12.5,
                        nbl=40, so=8, f0=12.0, global_cells=(1000, 1000, 500)):
    """Batched elastic gradients: ``nshots`` explosive-source shots on windows
    with nx, ny ~ U[size_range], nz fixed, at random offsets in the undulating
    10-layer model (velocity of the TTI batch recipe), vs = vp / 1.73 and
    Gardner density rho = 0.31 vp^0.25 (vp in m/s); source at the window
    centre 25 m deep; receivers every 4 cells at depth h.  Each entry is
    (true problem, starting problem): the starting vp (and vs, rho through
    the same relations) increases linearly with depth."""
    rng = np.random.default_rng(seed)
    gx, gy, gz = global_cells
    model = UndulatingTTI(seed, extent=(gx * h, gy * h, gz * h))
    dt = cfl_dt(h, model.vmax)

    def elastic(vp):
        vp = np.ascontiguousarray(vp, dtype=np.float32)
        return {"vp": vp, "vs": (vp / np.float32(1.73)).astype(np.float32),
                "rho": (0.31 * (vp.astype(np.float64) * 1000.0) ** 0.25).astype(np.float32)}

    shots = []
    for s in range(nshots):
        nx, ny = (int(v) for v in rng.integers(size_range[0], size_range[1] + 1, 2))
        ox = int(rng.integers(0, gx - nx + 1))
        oy = int(rng.integers(0, gy - ny + 1))
        m = elastic(model.window(ox, oy, nx, ny, nz, h)["vp"])
        src = np.array([[(nx // 2) * h, (ny // 2) * h, 25.0]], np.float32)
        rec = carpet_receivers(0.0, 0.0, 4 * h, (nx - 1) // 4 + 1, (ny - 1) // 4 + 1, h)
        wav = ricker(f0, dt, nt)[None, :]
        name = f"elastic-window-{nx}x{ny}x{nz}-at-{ox},{oy}-so{so}-nt{nt}"
        true = Problem(ELASTIC, nx, ny, nz, nbl, h, so, nt, dt, m, src, wav, rec, name=name)
        z = (np.arange(nz) / max(nz - 1, 1)).astype(np.float32)
        v0 = model.vmin + (model.vmax - model.vmin) * z
        start = elastic(np.broadcast_to(v0[None, None, :], (nx, ny, nz)))
        p0 = Problem(ELASTIC, nx, ny, nz, nbl, h, so, nt, dt, start, src, wav, rec,
                     name=name.replace("window", "window-start"))
        shots.append((true, p0))
    return shots
