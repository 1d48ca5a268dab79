"""Seeded synthetic inputs: meshes, physical parameters and initial states.

This module is shared by the CUDA path, the tests and the oracle.  It holds none of the
method's arithmetic (no residual, no solver, no FR operator): it only produces the
geometry nodes, the face list and an initial conservative state, and evaluates analytic
fields at point coordinates.

Mesh format (dict):
    d       spatial dimension (2 or 3)
    E       number of elements
    qg      geometry degree (1 or 2); geometry nodes sit on the Lobatto points {-1,(0),1}
    gnodes  float64 [E, (qg+1)^d, d], node a = a0 + (qg+1)*(a1 + (qg+1)*a2)
    faces   int32 [F, 6] rows (eL, fL, eR, fR, orient, bc); face f = 2*dir + side
            (side 0 at xi_dir = -1); eR = -1 marks a boundary face with bc 1 (far
            field) or 2 (no-slip adiabatic wall); orient as described in the C header.

The paper's meshes (sphere, cylinder with 5316 quadratic quads, SD7003) are not
available; the generators below stand in for them with the same character: quadratic
curved elements, periodic boxes, O-meshes with wall-normal stretching to aspect ratio
1e3, low Mach numbers.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = 1.4
PRANDTL = 0.72


# ----------------------------------------------------------------------------- meshes
def _lobatto(qg: int) -> np.ndarray:
    return np.array([-1.0, 1.0]) if qg == 1 else np.array([-1.0, 0.0, 1.0])


def box2d(nx: int, ny: int, Lx: float, Ly: float, qg: int = 2, warp: float = 0.0) -> dict:
    """Periodic [0,Lx]x[0,Ly] box of nx*ny quads; optional smooth periodic warp of the
    geometry nodes (amplitude `warp`, in units of the element size) makes the elements
    curved while keeping the mesh watertight and periodic."""
    hx, hy = Lx / nx, Ly / ny
    xi = _lobatto(qg)
    m = qg + 1
    E = nx * ny
    g = np.zeros((E, m * m, 2))
    for iy in range(ny):
        for ix in range(nx):
            e = ix + nx * iy
            for a1 in range(m):
                for a0 in range(m):
                    x = (ix + 0.5 * (xi[a0] + 1.0)) * hx
                    y = (iy + 0.5 * (xi[a1] + 1.0)) * hy
                    if warp:
                        s = math.sin(2 * math.pi * x / Lx) * math.sin(2 * math.pi * y / Ly)
                        t = math.sin(4 * math.pi * x / Lx) * math.cos(2 * math.pi * y / Ly)
                        x, y = x + warp * hx * s, y + warp * hy * (0.6 * s + 0.4 * t)
                    g[e, a0 + m * a1] = (x, y)
    faces = []
    for iy in range(ny):
        for ix in range(nx):
            e = ix + nx * iy
            faces.append((e, 1, (ix + 1) % nx + nx * iy, 0, 0, 0))
            faces.append((e, 3, ix + nx * ((iy + 1) % ny), 2, 0, 0))
    return dict(d=2, E=E, qg=qg, gnodes=g, faces=np.array(faces, dtype=np.int32),
                h_min=min(hx, hy), shape=(nx, ny), L=(Lx, Ly), kind="box2d")


def box3d(n: int, L: float, qg: int = 1) -> dict:
    """Periodic [0,L]^3 box of n^3 affine hexes."""
    h = L / n
    xi = _lobatto(qg)
    m = qg + 1
    E = n ** 3
    a = np.arange(m)
    A0, A1, A2 = np.meshgrid(a, a, a, indexing="ij")
    # node ordering a0 fastest
    A0, A1, A2 = A0.transpose(2, 1, 0).ravel(), A1.transpose(2, 1, 0).ravel(), A2.transpose(2, 1, 0).ravel()
    ex = np.arange(E) % n
    ey = (np.arange(E) // n) % n
    ez = np.arange(E) // (n * n)
    g = np.zeros((E, m ** 3, 3))
    g[:, :, 0] = (ex[:, None] + 0.5 * (xi[A0][None, :] + 1.0)) * h
    g[:, :, 1] = (ey[:, None] + 0.5 * (xi[A1][None, :] + 1.0)) * h
    g[:, :, 2] = (ez[:, None] + 0.5 * (xi[A2][None, :] + 1.0)) * h
    faces = []
    for iz in range(n):
        for iy in range(n):
            for ix in range(n):
                e = ix + n * (iy + n * iz)
                faces.append((e, 1, (ix + 1) % n + n * (iy + n * iz), 0, 0, 0))
                faces.append((e, 3, ix + n * ((iy + 1) % n + n * iz), 2, 0, 0))
                faces.append((e, 5, ix + n * (iy + n * ((iz + 1) % n)), 4, 0, 0))
    return dict(d=3, E=E, qg=qg, gnodes=g, faces=np.array(faces, dtype=np.int32),
                h_min=h, shape=(n, n, n), L=(L, L, L), kind="box3d")


def _stretch_ratio(h1: float, total: float, n: int) -> float:
    """geometric ratio s with h1 (s^n - 1)/(s - 1) = total"""
    lo, hi = 1.0 + 1e-12, 10.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if h1 * (mid ** n - 1.0) / (mid - 1.0) > total:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def omesh(nr: int, nt: int, r_in: float, r_out: float, h1: float, jitter: float = 0.0,
          seed: int = 0, qg: int = 2) -> dict:
    """O-mesh around a cylinder of radius r_in: nr radial x nt azimuthal quadratic quads,
    geometric radial stretching with first-cell height h1, optional seeded smooth jitter
    of the interior radial grid lines (fraction `jitter` of the local spacing).
    xi runs radially outward, eta counter-clockwise.  Wall (bc 2) at r_in, far field
    (bc 1) at r_out, periodic in the azimuth."""
    rng = np.random.default_rng(seed)
    s = _stretch_ratio(h1, r_out - r_in, nr)
    rb = r_in + h1 * (s ** np.arange(nr + 1) - 1.0) / (s - 1.0)
    rb[-1] = r_out
    dr = np.diff(rb)
    nh_t = 2 * nt if qg == 2 else nt
    th = 2 * math.pi * np.arange(nh_t) / nh_t                         # half-grid angles
    coef = rng.uniform(-1.0, 1.0, size=(nr + 1, 3, 2))

    def radius(j: int, theta: float) -> float:
        r = rb[j]
        if jitter and 0 < j < nr:
            f = sum(coef[j, k, 0] * math.sin((k + 1) * theta) + coef[j, k, 1] * math.cos((k + 1) * theta)
                    for k in range(3)) / 6.0
            r += jitter * min(dr[j - 1], dr[j]) * f
        return r

    m = qg + 1
    E = nr * nt
    g = np.zeros((E, m * m, 2))
    for it in range(nt):
        for ir in range(nr):
            e = ir + nr * it
            for a1 in range(m):
                ti = (qg * it + a1) % nh_t
                theta = th[ti]
                for a0 in range(m):
                    if qg == 2 and a0 == 1:
                        r = 0.5 * (radius(ir, theta) + radius(ir + 1, theta))
                    else:
                        r = radius(ir + (a0 // qg if qg == 2 else a0), theta)
                    g[e, a0 + m * a1] = (r * math.cos(theta), r * math.sin(theta))
    faces = []
    for it in range(nt):
        for ir in range(nr):
            e = ir + nr * it
            if ir + 1 < nr:
                faces.append((e, 1, e + 1, 0, 0, 0))
            else:
                faces.append((e, 1, -1, -1, 0, 1))
            if ir == 0:
                faces.append((e, 0, -1, -1, 0, 2))
            faces.append((e, 3, ir + nr * ((it + 1) % nt), 2, 0, 0))
    return dict(d=2, E=E, qg=qg, gnodes=g, faces=np.array(faces, dtype=np.int32),
                h_min=float(h1), shape=(nr, nt), r_in=r_in, r_out=r_out, kind="omesh")


# --------------------------------------------------------------- point coordinates
def gl_nodes(p: int) -> np.ndarray:
    """Gauss-Legendre nodes from numpy (used only to place initial-condition samples)."""
    return np.polynomial.legendre.leggauss(p + 1)[0]


def solution_point_coords(mesh: dict, p: int) -> np.ndarray:
    """Physical coordinates [d, Np, E] of the Gauss-Legendre points of every element,
    through the element's Lobatto geometry map (for sampling initial fields only)."""
    d, qg = mesh["d"], mesh["qg"]
    m = qg + 1
    x = gl_nodes(p)
    lob = _lobatto(qg)
    # Lagrange basis of the Lobatto nodes at x: B[t, a]
    B = np.ones((len(x), m))
    for a in range(m):
        for k in range(m):
            if k != a:
                B[:, a] *= (x - lob[k]) / (lob[a] - lob[k])
    gn = mesh["gnodes"]                                     # [E, m^d, d]
    if d == 2:
        G = gn.reshape(mesh["E"], m, m, 2)                  # [E, a1, a0, c]
        X = np.einsum("ia,jb,ebac->cjie", B, B, G)          # [c, j(eta), i(xi), E]
        return X.reshape(2, -1, mesh["E"])
    G = gn.reshape(mesh["E"], m, m, m, 3)                   # [E, a2, a1, a0, c]
    X = np.einsum("ia,jb,kc,ecbaz->zkjie", B, B, B, G)
    return X.reshape(3, -1, mesh["E"])


# ------------------------------------------------------------------------- fields
def freestream(d: int, mach: float, aoa: float = 0.0) -> np.ndarray:
    """rho = 1, |u| = 1, p = 1/(gamma Ma^2) (the paper's dimensionless impulsive start)."""
    p = 1.0 / (GAMMA * mach * mach)
    u = [math.cos(aoa), math.sin(aoa)] + ([0.0] if d == 3 else [])
    E = p / (GAMMA - 1.0) + 0.5 * sum(c * c for c in u)
    return np.array([1.0] + u + [E])


def prim_to_cons(rho, vel, p) -> np.ndarray:
    d = len(vel)
    ke = 0.5 * rho * sum(v * v for v in vel)
    return np.stack([rho] + [rho * v for v in vel] + [p / (GAMMA - 1.0) + ke])


def isentropic_vortex(X: np.ndarray, xc: float, yc: float, beta: float, mach: float,
                      Lx: float | None = None, Ly: float | None = None) -> np.ndarray:
    """Isentropic vortex of strength beta on rho = 1, u = (1, 0), T = p/rho = 1/(gamma Ma^2);
    exact solution of the Euler equations advected with the free stream.  With Lx, Ly
    the nearest periodic image is used."""
    x, y = X[0] - xc, X[1] - yc
    if Lx:
        x = x - Lx * np.round(x / Lx)
    if Ly:
        y = y - Ly * np.round(y / Ly)
    r2 = x * x + y * y
    Tinf = 1.0 / (GAMMA * mach * mach)
    f = np.exp(0.5 * (1.0 - r2))
    u = 1.0 - beta / (2 * math.pi) * f * y
    v = beta / (2 * math.pi) * f * x
    T = Tinf - (GAMMA - 1.0) * beta * beta / (8 * GAMMA * math.pi ** 2) * f * f
    rho = (T / Tinf) ** (1.0 / (GAMMA - 1.0))
    p = rho * T
    return prim_to_cons(rho, [u, v], p)


def taylor_green_box(mesh: dict, p: int, mach: float, noise_amp: float = 0.0, seed: int = 0,
                     kmax: int = 4) -> np.ndarray:
    """Taylor-Green field on a periodic box3d mesh with rho = 1, p0 = 1/(gamma Ma^2),
    plus seeded Fourier noise on each velocity component: the imaginary part of
    sum_k a_k exp(i phi_k) exp(i k.x) over wave vectors 1 <= |k|_inf <= kmax (one of each
    +-k pair), a_k ~ U(-1,1), phi_k ~ U(0, 2 pi), normalised to peak amplitude noise_amp.
    The box's Gauss-Legendre points form a tensor grid, so the sums factor per axis."""
    n = mesh["shape"][0]
    h = mesh["L"][0] / n
    xg = gl_nodes(p)
    npd = p + 1
    x1 = ((np.arange(n)[:, None] + 0.5 * (xg[None, :] + 1.0)) * h).ravel()   # index ex*npd + i
    x, y, z = np.meshgrid(x1, x1, x1, indexing="ij")
    u = np.sin(x) * np.cos(y) * np.cos(z)
    v = -np.cos(x) * np.sin(y) * np.cos(z)
    w = np.zeros_like(u)
    p0 = 1.0 / (GAMMA * mach * mach)
    pr = p0 + (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0) / 16.0
    if noise_amp:
        rng = np.random.default_rng(seed)
        K = kmax
        e1 = np.exp(1j * np.outer(np.arange(-K, K + 1), x1))            # [2K+1, N1]
        vel = [u, v, w]
        for comp in range(3):
            coef = np.zeros((K + 1, 2 * K + 1, 2 * K + 1), dtype=np.complex128)
            for a in range(0, K + 1):
                for b in range(-K, K + 1):
                    for c in range(-K, K + 1):
                        if max(abs(a), abs(b), abs(c)) < 1:
                            continue
                        if not (a > 0 or b > 0 or (b == 0 and c > 0)):
                            continue
                        coef[a, b + K, c + K] = rng.uniform(-1.0, 1.0) * np.exp(1j * rng.uniform(0.0, 2 * math.pi))
            W = np.einsum("abc,cz->abz", coef, e1)                      # [a, b, z]
            V = np.einsum("abz,by->ayz", W, e1)                         # [a, y, z]
            acc = np.einsum("ayz,ax->xyz", V, e1[K:])                   # [x, y, z]
            nz = acc.imag
            vel[comp] = vel[comp] + noise_amp * nz / np.max(np.abs(nz))
        u, v, w = vel
    fld = prim_to_cons(np.ones_like(x), [u, v, w], pr)                  # [5, X, Y, Z]
    fld = fld.reshape(5, n, npd, n, npd, n, npd)                        # v ex i0 ey i1 ez i2
    fld = fld.transpose(0, 6, 4, 2, 5, 3, 1)                            # v i2 i1 i0 ez ey ex
    return fld.reshape(5, npd ** 3, n ** 3)


def to_state(field: np.ndarray) -> np.ndarray:
    """[nv, Np, E] float64, C-contiguous (the library layout q[v][i][e])."""
    return np.ascontiguousarray(field, dtype=np.float64)


# ------------------------------------------------------------------------ configs
FLUXES = ("rusanov", "roe", "weiss_smith")


@dataclass
class Physics:
    gamma: float = GAMMA
    Pr: float = PRANDTL
    mu: float = 0.0
    eta: float = 2.0
    qinf: np.ndarray = field(default_factory=lambda: np.zeros(4))
    flux: str = "rusanov"          # inviscid common flux: "rusanov", "roe" or "weiss_smith"
    ws_umin: float = 1.0           # weiss_smith: floor of the reference velocity (free-stream units)

    @property
    def flux_code(self) -> int:
        return FLUXES.index(self.flux)

    def packed(self) -> np.ndarray:
        """gamma, Pr, mu, eta, qinf padded to 5, flux code (0 Rusanov, 1 Roe, 2 Roe with
        Weiss-Smith preconditioning), reference-velocity floor."""
        qi = np.zeros(5)
        qi[:len(self.qinf)] = self.qinf
        return np.concatenate([[self.gamma, self.Pr, self.mu, self.eta], qi,
                               [self.flux_code, self.ws_umin]]).astype(np.float64)


@dataclass
class Workload:
    name: str
    mesh: dict
    phys: Physics
    levels: list
    q0: np.ndarray
    dt: float = 0.0
    extra: dict = field(default_factory=dict)


def explicit_dt(mesh: dict, p: int, q: np.ndarray) -> float:
    """Reference explicit step h_min / ((2p+1) max(|u| + c)) (the paper leaves the CFL
    definition open; this is the reading used to size dt)."""
    d = mesh["d"]
    rho = q[0]
    vel = q[1:1 + d] / rho
    ke = 0.5 * rho * np.sum(vel * vel, axis=0)
    p_ = (GAMMA - 1.0) * (q[d + 1] - ke)
    c = np.sqrt(GAMMA * p_ / rho)
    smax = float(np.max(np.sqrt(np.sum(vel * vel, axis=0)) + c))
    return mesh["h_min"] / ((2 * p + 1) * smax)


def vortex2d(nx: int = 8, p: int = 2, levels=None, re: float = 100.0, mach: float = 0.5,
             L: float = 10.0, warp: float = 0.0, beta: float = 5.0) -> Workload:
    """2-D isentropic vortex on a periodic box (8x8 quads on [0,10]^2, p = 2, Re = 100,
    Ma = 0.5, strength 5: the small FP64 case; dt = 20x the explicit limit)."""
    mesh = box2d(nx, nx, L, L, qg=2, warp=warp)
    X = solution_point_coords(mesh, p)
    q0 = to_state(isentropic_vortex(X, L / 2, L / 2, beta, mach, L, L))
    phys = Physics(mu=1.0 / re if re else 0.0, qinf=freestream(2, mach))
    lv = levels if levels is not None else [p, p - 1]
    return Workload("vortex2d", mesh, phys, lv, q0, dt=20.0 * explicit_dt(mesh, p, q0))


def tgv3d(n: int = 32, p: int = 3, levels=None, re: float = 1600.0, mach: float = 0.1,
          noise: float = 1e-3, seed: int = 1) -> Workload:
    """3-D Taylor-Green field plus seeded Fourier noise on 32^3 periodic hexes, p = 3,
    Ma = 0.1, Re = 1600 (the throughput case)."""
    mesh = box3d(n, 2 * math.pi, qg=1)
    q0 = to_state(taylor_green_box(mesh, p, mach, noise, seed))
    phys = Physics(mu=1.0 / re, qinf=freestream(3, mach))
    lv = levels if levels is not None else [p, p - 1]
    return Workload("tgv3d", mesh, phys, lv, q0, dt=20.0 * explicit_dt(mesh, p, q0))


def cylinder_steady(nr: int = 64, nt: int = 128, p: int = 4, levels=None, mach: float = 1e-3,
                    re: float = 40.0, seed: int = 2) -> Workload:
    """Steady low-Mach cylinder: O-mesh 64x128, stretching to aspect ratio 1e3 at the wall,
    5% seeded jitter, p = 4, Ma = 1e-3, Re = 40, impulsive start."""
    h1 = (math.pi / nt) / 1e3
    mesh = omesh(nr, nt, 0.5, 20.0, h1, jitter=0.05, seed=seed)
    qinf = freestream(2, mach)
    q0 = to_state(np.broadcast_to(qinf[:, None, None], (4, (p + 1) ** 2, mesh["E"])).copy())
    phys = Physics(mu=1.0 / re, qinf=qinf)
    lv = levels if levels is not None else [4, 2, 1]
    return Workload("cylinder_steady", mesh, phys, lv, q0)


def cylinder_unsteady(nr: int = 96, nt: int = 192, p: int = 3, levels=None, mach: float = 0.05,
                      re: float = 150.0, seed: int = 4, cfl: float = 50.0) -> Workload:
    """Unsteady low-Mach vortex-shedding cylinder: O-mesh 96x192, first cell 0.01, p = 3,
    Ma = 0.05, Re = 150, seeded asymmetric perturbation; dt = CFL x explicit limit."""
    mesh = omesh(nr, nt, 0.5, 20.0, 0.01, jitter=0.0, seed=seed)
    X = solution_point_coords(mesh, p)
    qinf = freestream(2, mach)
    rng = np.random.default_rng(seed)
    amp, k = rng.uniform(0.02, 0.05), rng.uniform(0.5, 1.5)
    r2 = X[0] ** 2 + X[1] ** 2
    vpert = amp * np.exp(-((X[0] - 2.0) ** 2 + X[1] ** 2) / 4.0) * np.sin(k * X[0] + 0.3)
    rho = np.ones_like(r2)
    u = np.ones_like(r2)
    pinf = 1.0 / (GAMMA * mach * mach)
    q0 = to_state(prim_to_cons(rho, [u, vpert], pinf * np.ones_like(r2)))
    phys = Physics(mu=1.0 / re, qinf=qinf)
    lv = levels if levels is not None else [p, p - 1]
    return Workload("cylinder_unsteady", mesh, phys, lv, q0, dt=cfl * explicit_dt(mesh, p, q0))


def vortex_batch(nprob: int = 256, nmin: int = 4, nmax: int = 48, pmin: int = 1, pmax: int = 4, seed: int = 3,
                 re: float = 100.0, mach: float = 0.5, L: float = 10.0, cfl: float = 20.0):
    """Independent periodic [0, L]^2 isentropic-vortex problems of uneven size and degree:
    problem k has n_k x n_k quads with n_k ~ U{nmin..nmax}, p_k ~ U{pmin..pmax}, levels
    p{p-(p-1)} (a single level at p = 1), vortex centre (L/2, L/2) + U(-1, 1)^2 and strength
    U(4, 6), all seeded.  One dt for the whole batch: cfl x the smallest explicit limit.
    Returns (problems [(mesh, levels)], states, physics, dt)."""
    rng = np.random.default_rng(seed)
    problems, states, dts = [], [], []
    for _ in range(nprob):
        n = int(rng.integers(nmin, nmax + 1))
        p = int(rng.integers(pmin, pmax + 1))
        xc, yc = L / 2 + rng.uniform(-1, 1, size=2)
        beta = rng.uniform(4.0, 6.0)
        mesh = box2d(n, n, L, L, qg=2)
        X = solution_point_coords(mesh, p)
        q0 = to_state(isentropic_vortex(X, xc, yc, beta, mach, L, L))
        problems.append((mesh, [p, p - 1] if p > 1 else [1]))
        states.append(q0)
        dts.append(explicit_dt(mesh, p, q0))
    phys = Physics(mu=1.0 / re if re else 0.0, qinf=freestream(2, mach))
    return problems, states, phys, cfl * min(dts)
