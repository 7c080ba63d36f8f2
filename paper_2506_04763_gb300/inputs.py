"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This module only draws and lays out input data (grids, material fields,
initial states, boundary masks).  It holds none of the method's arithmetic.
It stands in for the paper's layered Cases 4/5, whose meshes and fields are
not published, with the workloads below.

Conventions (natural order, x fastest): vertex v = i + nx*(j + ny*k),
cell c = i + (nx-1)*(j + (ny-1)*k), state u[2v] = p_w (Pa), u[2v+1] = S_n.
Gravity points along -y in 2D and -z in 3D; the domain is the unit square or
cube; Dirichlet p_w sits on the top face.

Workloads:
  lens_square_2d         2D 33x33, sand with a 9x5-cell lens, h = 10 s, 4-level GMG.
  lognormal_cube_65      3D 65^3, lognormal K (ln K ~ N(ln 5e-11, 1), Gaussian
                         covariance, correlation length 8 cells, seed 1).
  lognormal_lenses_box   3D 257^3, lognormal K (seed 2) plus 6 random low-K lenses.
  ensemble_member        64 realisations (seeds 100..163) on 33^3, 49^3, 65^3, 97^3.
  dnapl_infiltration     3D 385^3, lognormal K (seed 3) plus lenses, NAPL inlet on top.
"""
import numpy as np

FLUIDS = dict(rho_w=1000.0, rho_n=1460.0, mu_w=1e-3, mu_n=9e-4)
GRAV = 9.81
SAND = dict(K=6.64e-11, phi=0.40, pd=755.0)
LENS = dict(K=3.32e-11, phi=0.39, pd=1163.0)
BROOKS_COREY = dict(S_wr=0.10, S_nr=0.0, lam=2.0)
P_TOP = 1e5


def grid(dim, nverts):
    if dim == 2:
        n = (int(nverts[0]), int(nverts[1]), 1)
    else:
        n = tuple(int(t) for t in nverts)
    h = tuple(1.0 / (t - 1) if t > 1 else 1.0 for t in n)
    g = (0.0, -GRAV, 0.0) if dim == 2 else (0.0, 0.0, -GRAV)
    return n, h, g


def ncells(dim, n):
    return (n[0] - 1) * (n[1] - 1) * ((n[2] - 1) if dim == 3 else 1)


def _coords(dim, n, h):
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    return (i.ravel() * h[0], j.ravel() * h[1], k.ravel() * (h[2] if dim == 3 else 0.0))


def top_mask(dim, n):
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    top = (j == n[1] - 1) if dim == 2 else (k == n[2] - 1)
    return top.ravel().astype(np.uint8)


def initial_state(dim, n, h, seed, noise=10.0, sn_amp=0.3, sn_width=0.05, sn_max=0.8):
    """Hydrostatic p_w (1e5 Pa on top) plus N(0, noise) Pa (not on the top
    face), and a NAPL blob S_n = amp exp(-r^2/width) around the top centre."""
    rng = np.random.default_rng(seed)
    x, y, z = _coords(dim, n, h)
    vert = y if dim == 2 else z
    pw = P_TOP + FLUIDS["rho_w"] * GRAV * (1.0 - vert) + rng.normal(0.0, noise, x.size)
    top = top_mask(dim, n).astype(bool)
    pw[top] = P_TOP
    if dim == 2:
        r2 = (x - 0.5) ** 2 + (y - 1.0) ** 2
    else:
        r2 = (x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 1.0) ** 2
    sn = np.clip(sn_amp * np.exp(-r2 / sn_width), 0.0, sn_max)
    u = np.empty(2 * x.size)
    u[0::2] = pw
    u[1::2] = sn
    return u


def lognormal_field(dim, n, seed, ell=8.0, mean=np.log(5e-11), sigma=1.0, rng=None):
    """ln K = mean + sigma * f, f a unit-variance stationary Gaussian field with
    covariance exp(-r^2/ell^2) (r in cells): white noise on a padded grid
    smoothed by a Gaussian of standard deviation ell/2 per axis, cropped and
    standardised."""
    from scipy import ndimage

    rng = np.random.default_rng(seed) if rng is None else rng
    shape = [(n[2] - 1) if dim == 3 else 1, n[1] - 1, n[0] - 1]
    pad = int(np.ceil(3 * ell))
    pshape = [s + 2 * pad if s > 1 else 1 for s in shape]
    w = rng.standard_normal(pshape)
    sig = [ell / 2.0 if s > 1 else 0.0 for s in shape]
    f = ndimage.gaussian_filter(w, sigma=sig, mode="wrap", truncate=4.0)
    sl = tuple(slice(pad, pad + s) if s > 1 else slice(0, 1) for s in shape)
    f = f[sl]
    sd = f.std()
    f = (f - f.mean()) / sd if sd > 0 else np.zeros_like(f)   # a single cell: the mean
    return np.exp(mean + sigma * f).ravel(), rng


def _lens_boxes(rng, dim, n, count, lo=8, hi=32):
    cshape = [n[0] - 1, n[1] - 1, (n[2] - 1) if dim == 3 else 1]
    boxes = []
    for _ in range(count):
        box = []
        for ax in range(dim):
            ext = int(rng.integers(lo, hi + 1))
            ext = min(ext, cshape[ax])
            start = int(rng.integers(0, cshape[ax] - ext + 1))
            box.append((start, start + ext))
        if dim == 2:
            box.append((0, 1))
        boxes.append(box)
    return boxes


def _paint(dim, n, arr, boxes, value=None, factor=None):
    cx, cy = n[0] - 1, n[1] - 1
    cz = (n[2] - 1) if dim == 3 else 1
    a = arr.reshape(cz, cy, cx)
    for (x0, x1), (y0, y1), (z0, z1) in boxes:
        if factor is not None:
            a[z0:z1, y0:y1, x0:x1] *= factor
        else:
            a[z0:z1, y0:y1, x0:x1] = value
    return a.ravel()


def problem(dim, nverts, K, phi, pd, u0, q_in=None, dirmask=None):
    n, h, g = grid(dim, nverts)
    nv = n[0] * n[1] * n[2]
    dm = top_mask(dim, n) if dirmask is None else np.ascontiguousarray(dirmask, np.uint8)
    pw_dir = np.where(dm.astype(bool), P_TOP, 0.0)
    prob = dict(dim=dim, n=n, h=h, g=g, K=np.ascontiguousarray(K, np.float64),
                phi=np.ascontiguousarray(phi, np.float64), pd=np.ascontiguousarray(pd, np.float64),
                dir=dm, pw_dir=pw_dir, q_in=q_in, u0=np.ascontiguousarray(u0, np.float64))
    prob.update(FLUIDS)
    prob.update(BROOKS_COREY)
    assert prob["K"].size == ncells(dim, n) and prob["u0"].size == 2 * nv
    return prob


def lens_square_2d():
    """2D 33x33 unit square, sand with a centred 9x5-cell lens (x-cells
    [11,20), y-cells [13,18)); state seed 0; one stage with h = 10 s."""
    dim, nv = 2, (33, 33)
    n, h, _ = grid(dim, nv)
    nc = ncells(dim, n)
    K = np.full(nc, SAND["K"])
    phi = np.full(nc, SAND["phi"])
    pd = np.full(nc, SAND["pd"])
    box = [[(11, 20), (13, 18), (0, 1)]]
    K = _paint(dim, n, K, box, LENS["K"])
    phi = _paint(dim, n, phi, box, LENS["phi"])
    pd = _paint(dim, n, pd, box, LENS["pd"])
    prob = problem(dim, nv, K, phi, pd, initial_state(dim, n, h, seed=0))
    prob.update(name="lens-square-2d-33x33", H=10.0, nlevels=4, smoother="jacobi")
    return prob


def lognormal_box(nvert, seed, lenses=0, name=None, ell=8.0):
    """3D box with lognormal K (seed) and optionally `lenses` random low-K
    lenses (extents U[8,32] cells per axis, K/20, p_d = 1163 Pa) drawn from the
    same generator after the field."""
    dim = 3
    nv = (nvert, nvert, nvert) if np.isscalar(nvert) else tuple(nvert)
    n, h, _ = grid(dim, nv)
    K, rng = lognormal_field(dim, n, seed, ell=ell)
    nc = K.size
    phi = np.full(nc, SAND["phi"])
    pd = np.full(nc, SAND["pd"])
    if lenses:
        boxes = _lens_boxes(rng, dim, n, lenses)
        K = _paint(dim, n, K, boxes, factor=1.0 / 20.0)
        pd = _paint(dim, n, pd, boxes, value=LENS["pd"])
    prob = problem(dim, nv, K, phi, pd, initial_state(dim, n, h, seed=seed))
    prob.update(name=name or ("box%d-seed%d" % (n[0], seed)), H=10.0)
    return prob


def levels_for(nvert):
    """Vertex-nested levels down to a coarsest grid of at most 5 vertices per axis
    (257 -> 7 levels, 385 -> 8, 97 -> 6, 65 -> 5, 49 -> 5, 33 -> 4)."""
    L, m = 1, int(nvert)
    while (m - 1) % 2 == 0 and m > 5:
        m = (m - 1) // 2 + 1
        L += 1
    return L


def lognormal_cube_65():
    p = lognormal_box(65, seed=1, name="lognormal-cube-65")
    p.update(nlevels=5, smoother="jacobi")
    return p


def lognormal_lenses_box(nvert=257):
    p = lognormal_box(nvert, seed=2, lenses=6, name="lognormal-lenses-%dcube" % nvert)
    p.update(nlevels=levels_for(nvert), smoother="gs8")
    return p


def ensemble_members():
    """(seed, vertices per axis) for the 64-realisation ensemble."""
    sizes = [33] * 16 + [49] * 16 + [65] * 16 + [97] * 16
    return list(zip(range(100, 164), sizes))


def ensemble_member(seed, nvert):
    p = lognormal_box(nvert, seed=seed, name="ens-%d-%d" % (seed, nvert))
    p.update(nlevels=levels_for(nvert), smoother="jacobi")
    return p


def dnapl_infiltration(nvert=385, inflow=0.1, half_width=0.05):
    """DNAPL infiltration: Neumann NAPL influx (kg m^-2 s^-1) through a top
    patch |x-.5|,|y-.5| <= half_width; Dirichlet p_w on the rest of the top."""
    p = lognormal_box(nvert, seed=3, lenses=6, name="dnapl-infiltration-%dcube" % nvert)
    dim, n, h = 3, p["n"], p["h"]
    x, y, z = _coords(dim, n, h)
    top = top_mask(dim, n).astype(bool)
    inlet = top & (np.abs(x - 0.5) <= half_width + 1e-12) & (np.abs(y - 0.5) <= half_width + 1e-12)
    i = np.rint(x / h[0]).astype(int)
    j = np.rint(y / h[1]).astype(int)
    ax = np.where((i == 0) | (i == n[0] - 1), 0.5, 1.0) * h[0]
    ay = np.where((j == 0) | (j == n[1] - 1), 0.5, 1.0) * h[1]
    q = np.zeros(2 * x.size)
    q[1::2] = np.where(inlet, inflow * ax * ay, 0.0)
    dm = (top & ~inlet).astype(np.uint8)
    p["q_in"] = q
    p["dir"] = dm
    p["pw_dir"] = np.where(dm.astype(bool), P_TOP, 0.0)
    p.update(nlevels=levels_for(nvert), smoother="gs8")
    return p


def random_problem(dim, nvert, seed, stress=False, dirichlet=True, gravity=True):
    """Small heterogeneous test problem: lognormal K (short correlation), a
    random lens with higher entry pressure, noisy hydrostatic p_w and a random
    S_n field.  With stress=True, S_n also takes values outside the physical
    range so that every clamp and cap branch of the laws is reached."""
    n, h, _ = grid(dim, nvert if dim == 3 else nvert[:2])
    rng = np.random.default_rng(seed)
    K, _ = lognormal_field(dim, n, seed, ell=2.0, rng=rng)
    nc = K.size
    phi = rng.uniform(0.3, 0.45, nc)
    pd = np.full(nc, SAND["pd"])
    boxes = _lens_boxes(rng, dim, n, 2, lo=2, hi=max(3, (n[0] - 1) // 2))
    pd = _paint(dim, n, pd, boxes, value=LENS["pd"])
    K = _paint(dim, n, K, boxes, factor=0.2)
    u = initial_state(dim, n, h, seed=seed + 1, noise=50.0)
    lo, hi = (-0.05, 1.0) if stress else (0.0, 0.6)
    u[1::2] = np.clip(u[1::2] + rng.uniform(0.0, 1.0, n[0] * n[1] * n[2]) * (hi - lo) + lo, lo, hi)
    dm = top_mask(dim, n) if dirichlet else np.zeros(n[0] * n[1] * n[2], np.uint8)
    prob = problem(dim, nvert if dim == 3 else nvert[:2], K, phi, pd, u, dirmask=dm)
    if not gravity:
        prob["g"] = (0.0, 0.0, 0.0)
    prob.update(name="random-%dd-%s-seed%d" % (dim, "x".join(map(str, n[:dim])), seed), H=10.0)
    return prob


# The layered Case-4 analogue (Sec. 6, Table case4): four horizontal layers,
# a light NAPL injected into the bottom layer at 0.05 pore volumes per year.
CASE4 = dict(K=(1e-13, 1e-12, 8e-13, 7e-13), phi=0.1, rho_w=1000.0, rho_n=700.0, mu_w=1e-3, mu_n=5.654e-5,
             S_wr=0.2, S_nr=0.1, lam=2.0, p_bottom=5e7, rate_pv_per_year=0.05)
YEAR = 365.0 * 86400.0


def case4_analogue(nverts=(129, 65), injecting=True):
    """Case 4's 500 m x 200 m vertical section (Table case4), with nverts
    vertices: four equal layers stacked in y (bottom first) with Case 4's
    permeabilities, p_d = 7.37 K^-0.43 Pa, Phi = 0.1 and its fluids and
    residual saturations, under this model's Brooks-Corey laws (Case 4's own
    k_r tables are not part of the model).  The state starts at S_w = 1 - S_nr
    (S_n = S_nr, immobile) with p_w hydrostatic from p_n = 5e7 Pa at the
    bottom, and p_w is held there (Dirichlet on the bottom row; Case 4 fixes
    p_n and S_w on that face).  NAPL enters through the vertices of the bottom
    layer's centre line with |x - 250 m| <= 25 m at 0.05 pore volumes per year
    (unit thickness) when `injecting`."""
    c = CASE4
    dim = 2
    n = (int(nverts[0]), int(nverts[1]), 1)
    Lx, Ly = 500.0, 200.0
    h = (Lx / (n[0] - 1), Ly / (n[1] - 1), 1.0)
    nc = ncells(dim, n)
    jc = (np.arange(nc) // (n[0] - 1))
    yc = (jc + 0.5) * h[1]
    layer = np.minimum((yc / Ly * 4).astype(int), 3)
    K = np.asarray(c["K"])[layer]
    pd = 7.37 * K ** -0.43
    phi = np.full(nc, c["phi"])
    nv = n[0] * n[1]
    x = (np.arange(nv) % n[0]) * h[0]
    jv = np.arange(nv) // n[0]
    y = jv * h[1]
    bottom = jv == 0
    # S_e = 1 everywhere: p_c = p_d of the vertex's lowest-entry-pressure cell
    # (the p_dmin of the interface condition), so p_w = p_n - p_c at the bottom
    pd_bottom = pd[layer == 0].max()
    pw = (c["p_bottom"] - pd_bottom) - c["rho_w"] * GRAV * y
    u = np.empty(2 * nv)
    u[0::2] = pw
    u[1::2] = c["S_nr"]
    q = np.zeros(2 * nv)
    if injecting:
        j_src = int(round(0.125 * Ly / h[1]))
        src = (jv == j_src) & (np.abs(x - 0.5 * Lx) <= 0.05 * Lx + 1e-9)
        rate = c["rho_n"] * c["phi"] * Lx * Ly * c["rate_pv_per_year"] / YEAR
        q[1::2] = np.where(src, rate / src.sum(), 0.0)
    prob = dict(dim=dim, n=n, h=h, g=(0.0, -GRAV, 0.0), K=K, phi=phi, pd=pd, dir=bottom.astype(np.uint8),
                pw_dir=np.where(bottom, pw, 0.0), q_in=q, u0=u, rho_w=c["rho_w"], rho_n=c["rho_n"], mu_w=c["mu_w"],
                mu_n=c["mu_n"], S_wr=c["S_wr"], S_nr=c["S_nr"], lam=c["lam"])
    prob.update(name="case4-analogue-%dx%d" % (n[0], n[1]), nlevels=levels_for(min(n[0], n[1])),
                smoother="gs8")
    return prob


# Case 1 (Sec. 6, Table case1): Buckley-Leverett displacement, p_c = 0.
CASE1 = dict(L=300.0, W=75.0, K=1e-7, phi=0.2, rho=1000.0, mu=1e-3, p_in=2e5, q_out=3e-4, T=1500 * 86400.0)


def case1_buckley_leverett(nx, ny=9):
    """Table case1's 300 m x 75 m strip with nx elements along x (ny vertices
    across, so that the multigrid hierarchy can coarsen), K = 1e-7 m^2,
    Phi = 0.2, equal densities and viscosities, S_wr = S_nr = 0, p_c = 0
    (p_d = 0), no gravity.  The model has no saturation Dirichlet condition,
    so the inlet column starts water-filled (S_n = 0, where k_rn = 0 keeps it
    so) with p_w = 2e5 Pa held (Dirichlet), and the outlet takes the table's
    NAPL outflow 3e-4 kg m^-2 s^-1 as a sink spread over its column by face
    share; everything else starts at S_n = 1.  Valid until the water front
    reaches the outlet (about 238 m at 1500 days)."""
    c = CASE1
    dim = 2
    n = (nx + 1, ny, 1)
    h = (c["L"] / nx, c["W"] / (ny - 1), 1.0)
    nc = nx * (ny - 1)
    nv = n[0] * n[1]
    i = np.arange(nv) % n[0]
    j = np.arange(nv) // n[0]
    u = np.empty(2 * nv)
    u[0::2] = c["p_in"]
    u[1::2] = np.where(i == 0, 0.0, 1.0)
    dm = (i == 0).astype(np.uint8)
    share = np.where((j == 0) | (j == ny - 1), 0.5, 1.0) * h[1]
    q = np.zeros(2 * nv)
    q[1::2] = np.where(i == nx, -c["q_out"] * share, 0.0)
    prob = dict(dim=dim, n=n, h=h, g=(0.0, 0.0, 0.0), K=np.full(nc, c["K"]), phi=np.full(nc, c["phi"]),
                pd=np.zeros(nc), dir=dm, pw_dir=np.where(i == 0, c["p_in"], 0.0), q_in=q, u0=u,
                rho_w=c["rho"], rho_n=c["rho"], mu_w=c["mu"], mu_n=c["mu"], S_wr=0.0, S_nr=0.0, lam=2.0)
    L, m = 1, list(n[:2])
    while all((t - 1) % 2 == 0 and t >= 3 for t in m):
        m = [(t - 1) // 2 + 1 for t in m]
        L += 1
    prob.update(name="case1-buckley-leverett-%d" % nx, nlevels=L, smoother="gs8")
    return prob


# Case 2 (Sec. 6, Table case2): extended Buckley-Leverett through two media,
# p_c = 0; each medium has its own polynomial relative permeabilities
# (rows {kind, a_w, n_w, a_n, b_n, c_n}: k_rw = a_w S_e^n_w, k_rn = a_n (1 -
# b_n S_e)^2 (1 - c_n S_e^2), kind 1 = polynomial).
CASE2 = dict(L=300.0, W=75.0, x_if=150.0, K1=1e-13, K2=1e-14, phi=0.2, rho=1000.0, mu_w=1e-3, mu_n=5e-3,
             p_in=2e5, q_out=2e-4, T=1500 * 86400.0,
             laws=((1.0, 1.831, 4.0, 0.75, 1.25, 1.652), (1.0, 0.4687, 2.0, 0.25, 1.25, 0.0)))


def case2_extended_buckley_leverett(nx, ny=9):
    """Table case2's 300 m x 75 m strip with nx elements along x (nx even, so
    that the media meet at a vertex line): medium 1 (x < 150 m) with K = 1e-13
    m^2 and the first pair of laws, medium 2 with K = 1e-14 m^2 and the
    second; Phi = 0.2, mu_w = 1e-3 and mu_n = 5e-3 Pa s, equal densities, no
    gravity, S_wr = S_nr = 0, p_d = 0.  The inlet and outlet are set up as in
    Case 1 (the inlet column water-filled with p_w = 2e5 Pa held, the outlet
    column taking the NAPL outflow 2e-4 kg m^-2 s^-1 by face share); valid
    while the water front is inside the strip (about 256 m at 1500 days)."""
    if nx % 2:
        raise ValueError("nx must be even")
    c = CASE2
    n = (nx + 1, ny, 1)
    h = (c["L"] / nx, c["W"] / (ny - 1), 1.0)
    nc = nx * (ny - 1)
    nv = n[0] * n[1]
    i = np.arange(nv) % n[0]
    j = np.arange(nv) // n[0]
    u = np.empty(2 * nv)
    u[0::2] = c["p_in"]
    u[1::2] = np.where(i == 0, 0.0, 1.0)
    xc = (np.arange(nc) % nx + 0.5) * h[0]
    law = (xc > c["x_if"]).astype(np.uint8)
    share = np.where((j == 0) | (j == ny - 1), 0.5, 1.0) * h[1]
    q = np.zeros(2 * nv)
    q[1::2] = np.where(i == nx, -c["q_out"] * share, 0.0)
    prob = dict(dim=2, n=n, h=h, g=(0.0, 0.0, 0.0), K=np.where(law == 0, c["K1"], c["K2"]),
                phi=np.full(nc, c["phi"]), pd=np.zeros(nc), dir=(i == 0).astype(np.uint8),
                pw_dir=np.where(i == 0, c["p_in"], 0.0), q_in=q, u0=u, rho_w=c["rho"], rho_n=c["rho"],
                mu_w=c["mu_w"], mu_n=c["mu_n"], S_wr=0.0, S_nr=0.0, lam=2.0,
                kr_laws=np.array(c["laws"]), cell_law=law)
    L, m = 1, list(n[:2])
    while all((t - 1) % 2 == 0 and t >= 3 for t in m):
        m = [(t - 1) // 2 + 1 for t in m]
        L += 1
    prob.update(name="case2-extended-buckley-leverett-%d" % nx, nlevels=L, smoother="gs8")
    return prob


def mixed_kr_laws(prob, seed):
    """A copy of `prob` whose cells draw (seeded) one of three relative
    permeability laws: Brooks-Corey, and the two polynomial laws of Case 2."""
    rng = np.random.default_rng(seed)
    out = dict(prob)
    out["kr_laws"] = np.array(((0.0, 0.0, 0.0, 0.0, 0.0, 0.0),) + CASE2["laws"])
    out["cell_law"] = rng.integers(0, 3, np.asarray(prob["K"]).size).astype(np.uint8)
    out["name"] = prob.get("name", "problem") + "-mixed-kr"
    return out

