"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the multigrid/IRK method itself: it builds
the coarsest input mesh (a structured triangulation of the unit square), the
analytic manufactured solution and its forcing (plain calculus, evaluated at
points the caller supplies), and reproducible pseudo-random numbers from the
published SplitMix64 generator.  Both sides consume these arrays; neither side
derives anything from the other.
"""
import numpy as np

__all__ = ["square_mesh", "cube_mesh", "mms3_velocity", "mms3_pressure", "mms3_forcing", "mms_velocity", "mms_pressure", "mms_forcing",
           "splitmix64", "uniform01", "normal", "random_vector", "wind_coefficients",
           "wind_field", "lid_velocity", "oseen_batch"]


def square_mesh(n):
    """Unit square, n x n squares, each cut by its (1,-1) diagonal into 2 triangles.

    Vertex (i, j) at (i/n, j/n) has id i + (n+1) j.  Square (i, j) gives the
    triangles [(i,j), (i+1,j), (i,j+1)] and [(i+1,j), (i+1,j+1), (i,j+1)].
    Returns (coords float64 [nv,2], cells int64 [nc,3], bnd uint8 [nv]) with
    bnd = 1 on every boundary vertex (the whole boundary is no-slip).
    """
    n = int(n)
    if n < 1:
        raise ValueError("n must be >= 1")
    ii, jj = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="xy")
    coords = np.stack([ii.ravel() / n, jj.ravel() / n], axis=1).astype(np.float64)
    vid = lambda i, j: i + (n + 1) * j
    cells = []
    for j in range(n):
        for i in range(n):
            cells.append([vid(i, j), vid(i + 1, j), vid(i, j + 1)])
            cells.append([vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)])
    cells = np.asarray(cells, dtype=np.int64)
    bi, bj = ii.ravel(), jj.ravel()
    bnd = ((bi == 0) | (bi == n) | (bj == 0) | (bj == n)).astype(np.uint8)
    return coords, cells, bnd


# ---------------------------------------------------------------------------
# Manufactured solution u = g(t) curl(psi), psi = sin^2(pi x) sin^2(pi y),
# p = g(t) sin(2 pi x) cos(2 pi y).  All derivatives are written out by hand.
# g = 1 (steady) or g = exp(-t).
# ---------------------------------------------------------------------------

def _g(t, kind):
    if kind == "steady":
        return 1.0, 0.0
    if kind == "exp":
        e = np.exp(-t)
        return e, -e
    raise ValueError(kind)


def mms_velocity(x, y, t=0.0, kind="steady"):
    """u = g(t) (d psi/dy, -d psi/dx); vanishes on the boundary of the unit square."""
    g, _ = _g(t, kind)
    sx, cx = np.sin(np.pi * x), np.cos(np.pi * x)
    sy, cy = np.sin(np.pi * y), np.cos(np.pi * y)
    ux = 2.0 * np.pi * sx * sx * sy * cy
    uy = -2.0 * np.pi * sx * cx * sy * sy
    return g * ux, g * uy


def mms_pressure(x, y, t=0.0, kind="steady"):
    """p = g(t) sin(2 pi x) cos(2 pi y); it has zero mean on the unit square."""
    g, _ = _g(t, kind)
    return g * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)


def mms_forcing(x, y, t=0.0, nu=1.0, kind="steady"):
    """f = g' u_s - nu g Lap(u_s) + g grad(p_s) for the fields above.

    With ux_s = pi sin^2(pi x) sin(2 pi y): Lap ux_s = 2pi^3 cos(2pi x) sin(2pi y)
    - 4 pi^3 sin^2(pi x) sin(2 pi y); uy_s = -pi sin(2 pi x) sin^2(pi y) gives
    Lap uy_s = 4 pi^3 sin(2pi x) sin^2(pi y) - 2 pi^3 sin(2 pi x) cos(2 pi y).
    """
    g, dg = _g(t, kind)
    pi = np.pi
    s2x, c2x = np.sin(2 * pi * x), np.cos(2 * pi * x)
    s2y, c2y = np.sin(2 * pi * y), np.cos(2 * pi * y)
    sx2 = np.sin(pi * x) ** 2
    sy2 = np.sin(pi * y) ** 2
    ux = pi * sx2 * s2y
    uy = -pi * s2x * sy2
    lap_ux = 2 * pi ** 3 * c2x * s2y - 4 * pi ** 3 * sx2 * s2y
    lap_uy = 4 * pi ** 3 * s2x * sy2 - 2 * pi ** 3 * s2x * c2y
    dpx = 2 * pi * c2x * c2y
    dpy = -2 * pi * s2x * s2y
    fx = dg * ux - nu * g * lap_ux + g * dpx
    fy = dg * uy - nu * g * lap_uy + g * dpy
    return fx, fy


# ---------------------------------------------------------------------------
# SplitMix64 (Steele, Lea, Flood 2014): state += 0x9E3779B97F4A7C15, then the
# published two multiply-xorshift rounds.  Vectorised over counters.
# ---------------------------------------------------------------------------
_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(seed, count, offset=0):
    """Return `count` uint64 outputs of SplitMix64 started from `seed`."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed, count, offset=0):
    """Doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed, count, offset=0):
    """Standard normals by Box-Muller on pairs of uniform01 draws."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m, offset)
    u1 = 1.0 - u[0::2]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
    return z[:count]


def random_vector(seed, count):
    """Seeded test vector with entries uniform in [-1, 1)."""
    return 2.0 * uniform01(seed, count) - 1.0


# ---------------------------------------------------------------------------
# Lid-driven cavity with a frozen wind (Oseen linearisation inputs)
# ---------------------------------------------------------------------------
def wind_coefficients(seed, kmax=4):
    """a_kl ~ N(0,1)/(k^2+l^2), k, l = 1..kmax (row-major), from SplitMix64."""
    z = normal(seed, kmax * kmax)
    k = np.arange(1, kmax + 1)
    return (z.reshape(kmax, kmax) / (k[:, None] ** 2 + k[None, :] ** 2))


def wind_field(x, y, a):
    """w = curl(psi), psi = sum a_kl sin(k pi x) sin(l pi y): w = (dpsi/dy, -dpsi/dx).
    Divergence-free and tangential-free on the unit square boundary."""
    kmax = a.shape[0]
    wx = np.zeros_like(x, dtype=np.float64)
    wy = np.zeros_like(x, dtype=np.float64)
    for k in range(1, kmax + 1):
        for l in range(1, kmax + 1):
            c = a[k - 1, l - 1]
            wx += c * l * np.pi * np.sin(k * np.pi * x) * np.cos(l * np.pi * y)
            wy -= c * k * np.pi * np.cos(k * np.pi * x) * np.sin(l * np.pi * y)
    return wx, wy


def lid_velocity(x, y):
    """u = (1, 0) on the lid y = 1 (corners excluded), 0 elsewhere."""
    on = (y == 1.0) & (x > 0.0) & (x < 1.0)
    return on.astype(np.float64), np.zeros_like(x, dtype=np.float64)


def oseen_batch(seed, count, sizes=(32, 64, 128, 256)):
    """Seeded description of a batch of independent Oseen stage systems:
    per system the mesh size n (uniform over `sizes`), Re ~ U[100, 1000]
    (nu = 1/Re), dt log-uniform in [1e-3, 1e-1] and a wind seed."""
    u = uniform01(seed, 4 * count).reshape(count, 4)
    out = []
    for i in range(count):
        n = sizes[min(int(u[i, 0] * len(sizes)), len(sizes) - 1)]
        re = 100.0 + 900.0 * u[i, 1]
        dt = 10.0 ** (-3.0 + 2.0 * u[i, 2])
        out.append({"n": n, "nu": 1.0 / re, "dt": dt, "wind_seed": int(seed * 1000 + i)})
    return out


# ---------------------------------------------------------------------------
# 3D inputs: Kuhn (6-tetrahedra-per-cube) mesh of the unit cube and the
# manufactured solution u = curl(psi (1,1,1)), psi = sin^2(pi x) sin^2(pi y)
# sin^2(pi z), p = sin(2 pi x) cos(2 pi y) cos(2 pi z).
# ---------------------------------------------------------------------------
def cube_mesh(n):
    """Unit cube, n^3 cubes, each cut into the 6 Kuhn tetrahedra: for every
    permutation sigma of the axes (lexicographic order), the tetrahedron with
    vertices 0, e_s1, e_s1 + e_s2, (1,1,1) (corner offsets of the cube).
    Vertex (i,j,k) has id i + (n+1) (j + (n+1) k).  bnd = 1 on the boundary."""
    import itertools
    n = int(n)
    r = np.arange(n + 1)
    K, J, I = np.meshgrid(r, r, r, indexing="ij")
    coords = np.stack([I.ravel() / n, J.ravel() / n, K.ravel() / n], axis=1).astype(np.float64)
    vid = lambda i, j, k: i + (n + 1) * (j + (n + 1) * k)
    cells = []
    perms = list(itertools.permutations(range(3)))
    for k in range(n):
        for j in range(n):
            for i in range(n):
                base = np.array([i, j, k])
                for sg in perms:
                    p = base.copy()
                    tet = [vid(*p)]
                    for ax in sg:
                        p = p.copy()
                        p[ax] += 1
                        tet.append(vid(*p))
                    cells.append(tet)
    cells = np.asarray(cells, dtype=np.int64)
    bi, bj, bk = I.ravel(), J.ravel(), K.ravel()
    bnd = ((bi == 0) | (bi == n) | (bj == 0) | (bj == n) | (bk == 0) | (bk == n)).astype(np.uint8)
    return coords, cells, bnd


def _s3(t):
    """S = sin^2(pi t) and its first three derivatives."""
    pi = np.pi
    return (np.sin(pi * t) ** 2, pi * np.sin(2 * pi * t), 2 * pi ** 2 * np.cos(2 * pi * t),
            -4 * pi ** 3 * np.sin(2 * pi * t))


def mms3_velocity(x, y, z):
    """u = (psi_y - psi_z, psi_z - psi_x, psi_x - psi_y); zero on the boundary."""
    Sx, Sy, Sz = _s3(x), _s3(y), _s3(z)
    px = Sx[1] * Sy[0] * Sz[0]
    py = Sx[0] * Sy[1] * Sz[0]
    pz = Sx[0] * Sy[0] * Sz[1]
    return py - pz, pz - px, px - py


def mms3_pressure(x, y, z):
    return np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) * np.cos(2 * np.pi * z)


def mms3_forcing(x, y, z, nu=1.0):
    """f = -nu Lap(u) + grad p with Lap(u) = curl(Lap(psi) (1,1,1))."""
    Sx, Sy, Sz = _s3(x), _s3(y), _s3(z)
    # d/dx, d/dy, d/dz of Lap(psi) = S''SS + SS''S + SSS''
    Lx = Sx[3] * Sy[0] * Sz[0] + Sx[1] * Sy[2] * Sz[0] + Sx[1] * Sy[0] * Sz[2]
    Ly = Sx[2] * Sy[1] * Sz[0] + Sx[0] * Sy[3] * Sz[0] + Sx[0] * Sy[1] * Sz[2]
    Lz = Sx[2] * Sy[0] * Sz[1] + Sx[0] * Sy[2] * Sz[1] + Sx[0] * Sy[0] * Sz[3]
    lap = (Ly - Lz, Lz - Lx, Lx - Ly)
    pi = np.pi
    s2x, c2x = np.sin(2 * pi * x), np.cos(2 * pi * x)
    s2y, c2y = np.sin(2 * pi * y), np.cos(2 * pi * y)
    s2z, c2z = np.sin(2 * pi * z), np.cos(2 * pi * z)
    gp = (2 * pi * c2x * c2y * c2z, -2 * pi * s2x * s2y * c2z, -2 * pi * s2x * c2y * s2z)
    return tuple(-nu * lap[d] + gp[d] for d in range(3))
