"""Seeded synthetic initial states (input generation only; none of the scheme's arithmetic).

Every generator returns ``(cfg, state)``:

* ``cfg``: dict with ndim, n, x0, x1, gamma, recon, riemann, rk, cfl, bc;
* ``state``: dict of float64 arrays in the library's external layout (no
  ghosts, x fastest): cell arrays rho, mx, my, mz, E of shape [nz][ny][nx];
  face fields b0 = Bx [nz][ny][nx+1], b1 = By [nz][ny+1][nx],
  b2 = Bz [nz+1][ny][nx] (3D) or the cell-centred Bz [1][ny][nx] (2D).

Face fields come from a discrete curl of an edge vector potential, so the
discrete divergence of B vanishes to round-off at t = 0; uniform field parts
are set on the faces directly.  Cell values of rho, v and p are point values at
cell centres.  The cell-centred field used for the energy is the mean of the
two bounding faces (2D Bz: the cell value).
"""
import functools
import math

import numpy as np

GAMMA = 5.0 / 3.0


def base_cfg(ndim, n, x0, x1, *, gamma=GAMMA, recon="plm", riemann="hlld", rk=2, cfl=0.4, bc="periodic",
             p_floor=0.0, emf="uct_hll"):
    if isinstance(bc, str):
        bc = [bc] * 6
    return {"ndim": ndim, "n": tuple(n), "x0": tuple(x0), "x1": tuple(x1), "gamma": gamma,
            "recon": recon, "riemann": riemann, "rk": rk, "cfl": cfl, "bc": list(bc), "p_floor": p_floor,
            "emf": emf}


def _grid(cfg):
    nd = cfg["ndim"]
    n = list(cfg["n"]) + [1] * (3 - len(cfg["n"]))
    if nd == 2:
        n[2] = 1
    x0 = list(cfg["x0"]) + [0.0] * (3 - len(cfg["x0"]))
    x1 = list(cfg["x1"]) + [1.0] * (3 - len(cfg["x1"]))
    dx = [(x1[d] - x0[d]) / n[d] for d in range(3)]
    return n, x0, dx


def cell_centres(cfg):
    """Arrays X, Y, Z of shape [nz][ny][nx] with the cell-centre coordinates."""
    n, x0, dx = _grid(cfg)
    xs = [x0[d] + (np.arange(n[d]) + 0.5) * dx[d] for d in range(3)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    return X, Y, Z


def _coords(cfg, stag):
    """Coordinates of a staggered location: stag[d] = 0 for cell centre, 1 for face/edge."""
    n, x0, dx = _grid(cfg)
    xs = []
    for d in range(3):
        if stag[d]:
            xs.append(x0[d] + np.arange(n[d] + 1) * dx[d])
        else:
            xs.append(x0[d] + (np.arange(n[d]) + 0.5) * dx[d])
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    return X, Y, Z


def faces_from_potential(cfg, Ax=None, Ay=None, Az=None):
    """Face field = discrete curl of an edge potential given as callables A(x, y, z).

    Ax lives on x-edges (x cell-centred, y and z on faces), and cyclically.
    In 2D only Az (at vertices) is used and the returned Bz is zero.
    """
    n, x0, dx = _grid(cfg)
    nd = cfg["ndim"]
    if nd == 2:
        X, Y, Z = _coords(cfg, (1, 1, 0))  # vertices, shape [1][ny+1][nx+1]
        az = Az(X, Y, Z) if Az is not None else np.zeros_like(X)
        bx = (az[:, 1:, :] - az[:, :-1, :]) / dx[1]            # [1][ny][nx+1]
        by = -(az[:, :, 1:] - az[:, :, :-1]) / dx[0]           # [1][ny+1][nx]
        return bx, by, np.zeros((1, n[1], n[0]))
    zero = lambda X, Y, Z: np.zeros_like(X)  # noqa: E731
    Ax = Ax or zero
    Ay = Ay or zero
    Az = Az or zero
    ax = Ax(*_coords(cfg, (0, 1, 1)))   # [nz+1][ny+1][nx]
    ay = Ay(*_coords(cfg, (1, 0, 1)))   # [nz+1][ny][nx+1]
    az = Az(*_coords(cfg, (1, 1, 0)))   # [nz][ny+1][nx+1]
    bx = (az[:, 1:, :] - az[:, :-1, :]) / dx[1] - (ay[1:, :, :] - ay[:-1, :, :]) / dx[2]   # [nz][ny][nx+1]
    by = (ax[1:, :, :] - ax[:-1, :, :]) / dx[2] - (az[:, :, 1:] - az[:, :, :-1]) / dx[0]   # [nz][ny+1][nx]
    bz = (ay[:, :, 1:] - ay[:, :, :-1]) / dx[0] - (ax[:, 1:, :] - ax[:, :-1, :]) / dx[1]   # [nz+1][ny][nx]
    return bx, by, bz


def cell_field(cfg, b0, b1, b2):
    """Cell-centred B (mean of bounding faces; 2D Bz is the cell value)."""
    bx = 0.5 * (b0[..., :-1] + b0[..., 1:])
    by = 0.5 * (b1[:, :-1, :] + b1[:, 1:, :])
    bz = 0.5 * (b2[:-1] + b2[1:]) if cfg["ndim"] == 3 else b2
    return bx, by, bz


def assemble(cfg, rho, vx, vy, vz, p, b0, b1, b2):
    """Conserved state from point primitives and face fields (Eq. Energy)."""
    bx, by, bz = cell_field(cfg, b0, b1, b2)
    g = cfg["gamma"]
    en = p / (g - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz) + 0.5 * (bx * bx + by * by + bz * bz)
    f = lambda a: np.ascontiguousarray(a, dtype=np.float64)  # noqa: E731
    return {"rho": f(rho), "mx": f(rho * vx), "my": f(rho * vy), "mz": f(rho * vz), "E": f(en),
            "b0": f(b0), "b1": f(b1), "b2": f(b2)}


def uniform_faces(cfg, B):
    n, _, _ = _grid(cfg)
    nx, ny, nz = n
    if cfg["ndim"] == 3:
        return (np.full((nz, ny, nx + 1), B[0]), np.full((nz, ny + 1, nx), B[1]), np.full((nz + 1, ny, nx), B[2]))
    return (np.full((1, ny, nx + 1), B[0]), np.full((1, ny + 1, nx), B[1]), np.full((1, ny, nx), B[2]))


# ---------------------------------------------------------------------------
# Paper and benchmark workloads
# ---------------------------------------------------------------------------

@functools.lru_cache(maxsize=16)
def _ot2d_unit_fields(n):
    """sin y, sin x at cell centres and the face field of A_z = cos y + cos 2x / 2
    on the n x n grid over [0, 2pi]^2 (unit amplitudes; read-only)."""
    cfg = base_cfg(2, (n, n), (0.0, 0.0), (2 * math.pi, 2 * math.pi))
    X, Y, _ = cell_centres(cfg)
    bx, by, _ = faces_from_potential(cfg, Az=lambda x, y, z: np.cos(y) + 0.5 * np.cos(2 * x))
    out = (np.sin(Y), np.sin(X), bx, by)
    for a in out:
        a.setflags(write=False)
    return out


def orszag_tang_2d(n=128, *, gamma=GAMMA, mach=1.0, beta=None, **kw):
    """2D Orszag-Tang vortex on [0, 2pi]^2: rho = G^2, p = G, v = M(-sin y, sin x),
    B = B0 (-sin y, sin 2x) from A_z = B0 (cos y + cos 2x / 2); B0 = 1 by default,
    or sqrt(2 G / beta) for a plasma beta (beta = 2 p / B0^2)."""
    cfg = base_cfg(2, (n, n), (0.0, 0.0), (2 * math.pi, 2 * math.pi), gamma=gamma, **kw)
    b0amp = 1.0 if beta is None else math.sqrt(2.0 * gamma / beta)
    siny, sinx, bxu, byu = _ot2d_unit_fields(n)
    rho = np.full(siny.shape, gamma * gamma)
    p = np.full(siny.shape, gamma)
    vx = -mach * siny
    vy = mach * sinx
    vz = np.zeros(siny.shape)
    bx = bxu * b0amp if b0amp != 1.0 else bxu.copy()
    by = byu * b0amp if b0amp != 1.0 else byu.copy()
    return cfg, assemble(cfg, rho, vx, vy, vz, p, bx, by, np.zeros((1, n, n)))


def orszag_tang_3d(n=(64, 64, 64), **kw):
    """3D Orszag-Tang of §4.1 (unit periodic cube, rho = 25/9, p = 5/3,
    v = (-zeta sin 2pi y, zeta sin 2pi x, 0.2 sin 2pi z), zeta = 1 + sin(2pi z)/5,
    B = (-sin 2pi y, sin 4pi x, 0) from A_z = cos(2pi y)/(2pi) + cos(4pi x)/(4pi))."""
    if isinstance(n, int):
        n = (n, n, n)
    cfg = base_cfg(3, n, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), **kw)
    X, Y, Z = cell_centres(cfg)
    tp = 2 * math.pi
    zeta = 1.0 + np.sin(tp * Z) / 5.0
    rho = np.full_like(X, 25.0 / 9.0)
    p = np.full_like(X, 5.0 / 3.0)
    vx = -zeta * np.sin(tp * Y)
    vy = zeta * np.sin(tp * X)
    vz = 0.2 * np.sin(tp * Z)
    bx, by, bz = faces_from_potential(cfg, Az=lambda x, y, z: np.cos(tp * y) / tp + np.cos(2 * tp * x) / (2 * tp))
    return cfg, assemble(cfg, rho, vx, vy, vz, p, bx, by, bz)


def gaussian_field(shape, rng, kmin=1.0, kmax=8.0):
    """Real random field with i.i.d. N(0,1) complex Fourier coefficients on the
    integer wavevectors kmin <= |k| <= kmax, Hermitian by construction (inverse
    real FFT), normalised to unit rms."""
    nd = len(shape)
    freqs = [np.fft.fftfreq(s, d=1.0 / s) for s in shape[:-1]] + [np.fft.rfftfreq(shape[-1], d=1.0 / shape[-1])]
    K = np.meshgrid(*freqs, indexing="ij")
    kk = np.sqrt(sum(k * k for k in K))
    mask = (kk >= kmin) & (kk <= kmax)
    coef = (rng.standard_normal(kk.shape) + 1j * rng.standard_normal(kk.shape)) * mask
    f = np.fft.irfftn(coef, s=shape, axes=tuple(range(nd)))
    return f / np.sqrt(np.mean(f * f))


def turbulent_3d(n=256, *, seed=20251120, amp=0.01, kmax=8.0, **kw):
    """3D periodic unit cube: rho = 1 + 0.01 g_rho, p = 1, v = 0.01 (g_x, g_y, g_z),
    uniform B = (1, 1, 1)/sqrt 3; g_* Gaussian random fields with 1 <= |k| <= 8."""
    if isinstance(n, int):
        n = (n, n, n)
    cfg = base_cfg(3, n, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), **kw)
    rng = np.random.default_rng(seed)
    shape = (n[2], n[1], n[0])
    rho = 1.0 + amp * gaussian_field(shape, rng, kmax=kmax)
    vx = amp * gaussian_field(shape, rng, kmax=kmax)
    vy = amp * gaussian_field(shape, rng, kmax=kmax)
    vz = amp * gaussian_field(shape, rng, kmax=kmax)
    p = np.ones(shape)
    s = 1.0 / math.sqrt(3.0)
    bx, by, bz = uniform_faces(cfg, (s, s, s))
    return cfg, assemble(cfg, rho, vx, vy, vz, p, bx, by, bz)


def blast_3d(n=512, *, recon="wenoz", rk=3, p_floor=1e-12, bc="outflow", **kw):
    """Magnetised blast on [-1/2, 1/2]^3 with outflow boundaries: rho = 1,
    p = 0.1 outside and 10 for cell centres with r <= 0.1, v = 0,
    uniform B = (10/sqrt 2, 10/sqrt 2, 0).  At plasma beta 0.002 the recovered
    pressure (E minus a magnetic energy 500 times the thermal one) turns
    negative within a few steps at every resolution, so this workload uses the
    pressure floor 1e-12 on the recovered primitives."""
    if isinstance(n, int):
        n = (n, n, n)
    cfg = base_cfg(3, n, (-0.5, -0.5, -0.5), (0.5, 0.5, 0.5), recon=recon, rk=rk, bc=bc, p_floor=p_floor, **kw)
    X, Y, Z = cell_centres(cfg)
    r = np.sqrt(X * X + Y * Y + Z * Z)
    rho = np.ones_like(X)
    p = np.where(r <= 0.1, 10.0, 0.1)
    z0 = np.zeros_like(X)
    b = 10.0 / math.sqrt(2.0)
    bx, by, bz = uniform_faces(cfg, (b, b, 0.0))
    return cfg, assemble(cfg, rho, z0, z0, z0, p, bx, by, bz)


def cpa_3d(n=32, *, eps=0.1, rho0=1.0, p0=0.1, sign=+1.0, t=0.0, **kw):
    """Circularly polarised Alfven wave of §4.2 on the unit periodic cube,
    k = 2 pi (1, 1, 1).  In the frame e1 = k/|k|, e2, e3 (right-handed):
    B = e1 + eps (sin phi e2 + cos phi e3), v = sign * eps (sin phi e2 + cos phi e3),
    phi = k.x (reading: the second velocity term is along e3).  With B_par = 1 and
    rho0 = 1 the Alfven speed is 1; sign = +1 travels along -e1.  A nonzero t
    gives the exact solution translated by the Alfven speed."""
    if isinstance(n, int):
        n = (n, n, n)
    cfg = base_cfg(3, n, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), **kw)
    return cfg, _cpa_state(cfg, eps, rho0, p0, sign, t, np.array([1.0, 1.0, 1.0]))


def cpa_2d(n=32, *, eps=0.1, rho0=1.0, p0=0.1, sign=+1.0, t=0.0, **kw):
    """2D analogue of the circularly polarised wave, k = 2 pi (1, 1) on the unit square."""
    cfg = base_cfg(2, (n, n), (0.0, 0.0), (1.0, 1.0), **kw)
    return cfg, _cpa_state(cfg, eps, rho0, p0, sign, t, np.array([1.0, 1.0, 0.0]))


def _cpa_frame(kdir):
    e1 = kdir / np.linalg.norm(kdir)
    tmp = np.array([0.0, 0.0, 1.0]) if abs(e1[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    if np.allclose(kdir, [1, 1, 0]):
        e3 = np.array([0.0, 0.0, 1.0])
        e2 = np.cross(e3, e1)
    else:
        e2 = np.cross(tmp, e1)
        e2 /= np.linalg.norm(e2)
        e3 = np.cross(e1, e2)
    return e1, e2, e3


def _cpa_state(cfg, eps, rho0, p0, sign, t, kdir):
    e1, e2, e3 = _cpa_frame(kdir)
    kvec = 2 * math.pi * kdir
    kmag = np.linalg.norm(kvec)
    va = 1.0 / math.sqrt(rho0)
    # travelling along -sign*e1: phi(x, t) = k.x + sign*|k| va t
    shift = sign * kmag * va * t

    def phase(x, y, z):
        return kvec[0] * x + kvec[1] * y + kvec[2] * z + shift

    X, Y, Z = cell_centres(cfg)
    ph = phase(X, Y, Z)
    dv = [eps * (np.sin(ph) * e2[d] + np.cos(ph) * e3[d]) for d in range(3)]
    vx, vy, vz = (sign * va * dv[0], sign * va * dv[1], sign * va * dv[2])
    rho = np.full_like(X, rho0)
    p = np.full_like(X, p0)
    # transverse field from the potential A = (eps/|k|)(sin phi e2 + cos phi e3)
    a = eps / kmag
    if cfg["ndim"] == 3:
        pots = [lambda x, y, z, d=d: a * (np.sin(phase(x, y, z)) * e2[d] + np.cos(phase(x, y, z)) * e3[d])
                for d in range(3)]
        bx, by, bz = faces_from_potential(cfg, Ax=pots[0], Ay=pots[1], Az=pots[2])
        ux, uy, uz = uniform_faces(cfg, e1)
        bx, by, bz = bx + ux, by + uy, bz + uz
    else:
        # 2D: in-plane part from A_z; Bz (cell) = eps cos(phi) e3_z at cell centres
        bx, by, _ = faces_from_potential(
            cfg, Az=lambda x, y, z: a * (np.sin(phase(x, y, z)) * e2[2] + np.cos(phase(x, y, z)) * e3[2]))
        ux, uy, _ = uniform_faces(cfg, e1)
        bx, by = bx + ux, by + uy
        bz = eps * (np.sin(ph) * e2[2] + np.cos(ph) * e3[2])
    return assemble(cfg, rho, vx, vy, vz, p, bx, by, bz)


def ensemble_members(count=256, *, seed=4, sizes=(64, 96, 128, 192, 256, 384, 512), gamma=GAMMA):
    """Batched ensemble parameters: grid size uniform over `sizes`, plasma beta
    in [0.1, 10] and Mach in [0.5, 3] log-uniform, drawn from one seeded stream."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(sizes[rng.integers(len(sizes))])
        beta = float(math.exp(rng.uniform(math.log(0.1), math.log(10.0))))
        mach = float(math.exp(rng.uniform(math.log(0.5), math.log(3.0))))
        out.append({"n": n, "beta": beta, "mach": mach})
    return out


def ensemble_member_state(m, **kw):
    """Orszag-Tang member with rho = G^2, p = G (sound speed 1), v0 = Mach, B0 = sqrt(2G/beta)."""
    return orszag_tang_2d(m["n"], mach=m["mach"], beta=m["beta"], **kw)


def adjoint_2d(n=256, *, seed=5, amp=0.05, kmax=6.0, **kw):
    """2D periodic unit square: rho = 1 + 0.05 g_rho, v = 0.05 (g_x, g_y, 0), p = 1,
    uniform B = (1, 0.5, 0); Gaussian random fields with 1 <= |k| <= 6."""
    cfg = base_cfg(2, (n, n), (0.0, 0.0), (1.0, 1.0), **kw)
    rng = np.random.default_rng(seed)
    shape = (n, n)
    rho = (1.0 + amp * gaussian_field(shape, rng, kmax=kmax))[None]
    vx = (amp * gaussian_field(shape, rng, kmax=kmax))[None]
    vy = (amp * gaussian_field(shape, rng, kmax=kmax))[None]
    vz = np.zeros_like(rho)
    p = np.ones_like(rho)
    bx, by, bz = uniform_faces(cfg, (1.0, 0.5, 0.0))
    return cfg, assemble(cfg, rho, vx, vy, vz, p, bx, by, bz)


def to_glm(cfg, st, alpha=0.1):
    """The same initial state for the scheme with GLM divergence cleaning:
    cell-centred field = mean of the two faces (2D B_z: the cell value),
    psi = 0.  Returns (cfg with divb = glm, state with the GLM keys)."""
    bx, by, bz = cell_field(cfg, st["b0"], st["b1"], st["b2"])
    out = {k: st[k] for k in ("rho", "mx", "my", "mz", "E")}
    out.update(bx=np.ascontiguousarray(bx), by=np.ascontiguousarray(by), bz=np.ascontiguousarray(bz),
               psi=np.zeros_like(bx))
    return dict(cfg, divb="glm", glm_alpha=alpha), out


def smooth_2d(n=16, *, seed=5, bpert=0.0):
    """Smooth 2D periodic state on the unit square with no exactly tied limiter
    or min/max decision (a field constant along an axis ties minmod(0, 0),
    where the scheme is only directionally differentiable): Gaussian random
    rho, vx, vy (5 %, |k| <= 3), and vz, p and the cell B_z varying along both
    axes; in-plane face field (1, 0.5), plus, for bpert > 0, the curl of the
    periodic potential A_z = bpert/(2 pi) sin(2 pi x + 0.3) sin(2 pi y + 1.1)
    (without it the face field is uniform, so derivatives with respect to the
    initial face field meet minmod(0, 0) in the edge reconstruction).
    Returns (cfg, state, prims)."""
    cfg = base_cfg(2, (n, n), (0, 0), (1, 1))
    rng = np.random.default_rng(seed)
    X, Y, _ = cell_centres(cfg)
    tp = 2 * np.pi
    prim = {"rho": 1 + 0.05 * gaussian_field((n, n), rng, kmax=3.0)[None],
            "vx": 0.05 * gaussian_field((n, n), rng, kmax=3.0)[None],
            "vy": 0.05 * gaussian_field((n, n), rng, kmax=3.0)[None],
            "vz": 0.03 * np.sin(tp * X + 1.0) * np.cos(tp * Y + 0.4),
            "p": 1 + 0.05 * np.cos(tp * (X + 2 * Y) + 0.7)}
    bx, by, _ = uniform_faces(cfg, (1.0, 0.5, 0.0))
    if bpert > 0.0:
        px, py, _ = faces_from_potential(
            cfg, Az=lambda x, y, z: bpert / tp * np.sin(tp * x + 0.3) * np.sin(tp * y + 1.1))
        bx, by = bx + px, by + py
    bz = 0.2 + 0.1 * np.sin(tp * (2 * X + Y) + 0.3)
    st = assemble(cfg, prim["rho"], prim["vx"], prim["vy"], prim["vz"], prim["p"], bx, by, bz)
    return cfg, st, prim


def random_state(cfg, seed, *, rho=(0.5, 1.5), v=0.5, p=(0.5, 1.5), bamp=0.5, b0=(0.3, -0.2, 0.25)):
    """White-noise state for parity checks: uniform-random rho, v, p per cell and a
    random edge potential plus a uniform field, so div B = 0 discretely and every
    limiter and wave-fan branch is exercised."""
    rng = np.random.default_rng(seed)
    n, x0, dx = _grid(cfg)
    shape = (n[2], n[1], n[0])
    r = rng.uniform(*rho, size=shape)
    vx = rng.uniform(-v, v, size=shape)
    vy = rng.uniform(-v, v, size=shape)
    vz = rng.uniform(-v, v, size=shape)
    pp = rng.uniform(*p, size=shape)
    ux, uy, uz = uniform_faces(cfg, b0)
    if cfg["ndim"] == 3:
        # periodic random potentials on edges (index-periodic so faces are periodic)
        ax = rng.standard_normal((n[2], n[1], n[0])) * bamp * dx[1]
        ay = rng.standard_normal((n[2], n[1], n[0])) * bamp * dx[0]
        az = rng.standard_normal((n[2], n[1], n[0])) * bamp * dx[0]
        wrapz = lambda a: np.concatenate([a, a[:1]], axis=0)  # noqa: E731
        wrapy = lambda a: np.concatenate([a, a[:, :1]], axis=1)  # noqa: E731
        wrapx = lambda a: np.concatenate([a, a[:, :, :1]], axis=2)  # noqa: E731
        AX = wrapz(wrapy(ax))            # [nz+1][ny+1][nx]
        AY = wrapz(wrapx(ay))            # [nz+1][ny][nx+1]
        AZ = wrapy(wrapx(az))            # [nz][ny+1][nx+1]
        bx = (AZ[:, 1:, :] - AZ[:, :-1, :]) / dx[1] - (AY[1:, :, :] - AY[:-1, :, :]) / dx[2]
        by = (AX[1:, :, :] - AX[:-1, :, :]) / dx[2] - (AZ[:, :, 1:] - AZ[:, :, :-1]) / dx[0]
        bz = (AY[:, :, 1:] - AY[:, :, :-1]) / dx[0] - (AX[:, 1:, :] - AX[:, :-1, :]) / dx[1]
        bx, by, bz = bx + ux, by + uy, bz + uz
    else:
        az = rng.standard_normal((1, n[1], n[0])) * bamp * dx[0]
        AZ = np.concatenate([az, az[:, :1]], axis=1)
        AZ = np.concatenate([AZ, AZ[:, :, :1]], axis=2)  # [1][ny+1][nx+1]
        bx = (AZ[:, 1:, :] - AZ[:, :-1, :]) / dx[1] + ux
        by = -(AZ[:, :, 1:] - AZ[:, :, :-1]) / dx[0] + uy
        bz = rng.uniform(-bamp, bamp, size=(1, n[1], n[0])) + b0[2]
    return assemble(cfg, r, vx, vy, vz, pp, bx, by, bz)
