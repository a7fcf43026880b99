"""Seeded synthetic problem descriptions shared by the CUDA path and the oracle.

This module holds no arithmetic of the method: it only describes problems
(grid, degree, geometry parameters, material data, boundary data) and draws
the random numbers a problem needs (void centres and radii, ellipsoid axes and
rotations, test vectors).  Random geometry is drawn with splitmix64 (Steele,
Lea and Flood, "Fast splittable pseudorandom number generators", 2014) so the
same descriptor is reproduced bit for bit on every machine.

A problem is a plain dict so it can be serialised, printed and handed both to
the C-ABI binding and to the oracle.

Keys
----
dim, cells, lo, hi, p       grid: d, cells per axis, box corners, degree
pde                         "poisson" | "elasticity"
kappa                       Poisson conductivity in the physical domain
E, nu                       elasticity (isotropic, Voigt notation)
alpha, beta                 fictitious-domain factor and penalty parameter
geometry                    {"kind": "none"|"ball"|"voids"|"ellipsoid", ...}
source                      {"kind": "const", "f0"} | {"kind": "sin3"} |
                            {"kind": "square_mms", "a", "kappa"}
dirichlet                   {"kind": "levelset"|"faces"|"none",
                             "g": "zero"|"sin3"|"square_mms", "faces": [...]}
traction                    {"face": id, "t": (tx, ty, tz)} or None
quad_depth                  space-tree depth for cut cells
omega, n_pre, n_post        smoother settings (omega None: paper default)
coarse_cells                h-coarsening stops once every axis has at most
                            this many cells
overlay_levels              multi-level hp refinement depth K (0: uniform)
smoother                    "elementwise" | "patchwise" | "jacobi" | "gauss_seidel"
space, drop_outside         "tensor" | "trunk" elements; remove fully fictitious
                            cells (oracle only)
"""
from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64_next(state: int) -> tuple[int, int]:
    """One splitmix64 step: returns (new_state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    z = z ^ (z >> 31)
    return state, z


class SplitMix64:
    """Deterministic stream of uniform doubles in [0, 1) (53-bit)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state, out = splitmix64_next(self.state)
        return out

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        u = (self.next_u64() >> 11) * (1.0 / (1 << 53))
        return lo + (hi - lo) * u

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] inclusive."""
        return lo + int(self.next_u64() % (hi - lo + 1))


def instance_seed(base: int, i: int) -> int:
    """Seed of instance i of a batch: one splitmix64 output of base ^ i."""
    _, out = splitmix64_next((base ^ (i * 0x632BE59BD9B4E019)) & MASK64)
    return out


# --------------------------------------------------------------------------
# problem descriptors
# --------------------------------------------------------------------------

def _base(dim, cells, p, **kw):
    d = dict(dim=dim, cells=tuple(cells), lo=(0.0,) * dim, hi=(1.0,) * dim, p=p,
             pde="poisson", kappa=1.0, E=1.0, nu=0.3, alpha=1e-8, beta=1e4,
             geometry=dict(kind="none"), source=dict(kind="const", f0=1.0),
             dirichlet=dict(kind="none"), traction=None, quad_depth=3,
             omega=None, n_pre=5, n_post=5, coarse_cells=4)
    d.update(kw)
    return d


def poisson2d_circle(cells=16, p=2, alpha=1e-6, radius=0.4, quad_depth=3):
    """2D Poisson on the unit square embedding a circle of radius 0.4,
    f = 1, homogeneous Dirichlet on the circle by penalty (16x16, p=2)."""
    return _base(2, (cells, cells), p, alpha=alpha, beta=1e4,
                 geometry=dict(kind="ball", center=(0.5, 0.5), radius=radius),
                 source=dict(kind="const", f0=1.0),
                 dirichlet=dict(kind="levelset", g="zero"), quad_depth=quad_depth,
                 name=f"poisson2d_circle_{cells}x{cells}_p{p}")


def poisson3d_sphere(cells=32, p=3, alpha=1e-8, radius=0.45, quad_depth=3):
    """3D Poisson on the unit cube embedding a sphere r=0.45 (32^3, p=3),
    manufactured solution u = sin(pi x) sin(pi y) sin(pi z): f = 3 pi^2 u and
    g_D = u on the sphere by penalty."""
    return _base(3, (cells,) * 3, p, alpha=alpha, beta=1e4,
                 geometry=dict(kind="ball", center=(0.5, 0.5, 0.5), radius=radius),
                 source=dict(kind="sin3"),
                 dirichlet=dict(kind="levelset", g="sin3"), quad_depth=quad_depth,
                 name=f"poisson3d_sphere_{cells}^3_p{p}")


def square_mms(cells=8, p=2, kappa=10.0, beta=1e4, alpha=1e-8):
    """Mesh-fitting (psi = 0) rotated-square Poisson problem: unit square,
    u = cos(a x') sin(a y') / (2 kappa a^2), a = 3 pi / 2, x' = x - 1/2,
    y' = y - 1/2, source cos(a x') sin(a y'), Dirichlet u on all four edges by
    penalty."""
    a = 1.5 * math.pi
    return _base(2, (cells, cells), p, kappa=kappa, alpha=alpha, beta=beta,
                 geometry=dict(kind="none"),
                 source=dict(kind="square_mms", a=a, kappa=kappa),
                 dirichlet=dict(kind="faces", g="square_mms", faces=[0, 1, 2, 3]),
                 quad_depth=0, name=f"square_mms_{cells}x{cells}_p{p}")


def rotated_square(cells=12, p=2, psi_deg=30.0, kappa=10.0, beta=1e4, alpha=1e-8):
    """Immersed rotating-square Poisson problem (Sec. 4.1.2): the unit square
    centred at (1/2, 1/2) rotated by psi, in the fixed background box
    [-1/4, 5/4]^2 that holds every rotation (12 cells per axis: h = 1/8);
    u = cos(a x') sin(a y') / (2 kappa a^2) in the rotated coordinates,
    a = 3 pi / 2, source cos(a x') sin(a y'), Dirichlet u on the square's
    edges by penalty."""
    a = 1.5 * math.pi
    ang = math.radians(psi_deg)
    return _base(2, (cells, cells), p, lo=(-0.25, -0.25), hi=(1.25, 1.25), kappa=kappa,
                 alpha=alpha, beta=beta,
                 geometry=dict(kind="rotated_square", center=(0.5, 0.5), half=0.5, angle=ang),
                 source=dict(kind="square_mms", a=a, kappa=kappa, angle=ang),
                 dirichlet=dict(kind="levelset", g="square_mms"),
                 name=f"rotated_square_{cells}x{cells}_p{p}_psi{psi_deg:g}")


def draw_voids(n_voids=64, rmin=0.03, rmax=0.08, gap=1.0 / 64, seed=0, max_tries=100000):
    """Void centres and radii for the perforated block: radii U[rmin, rmax],
    centres uniform in the unit cube, rejection keeps a gap between voids and
    from the box faces.  Returns an (n, 4) array of (cx, cy, cz, r)."""
    rng = SplitMix64(seed)
    out = []
    tries = 0
    while len(out) < n_voids:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("void sampler did not converge")
        r = rng.uniform(rmin, rmax)
        c = [rng.uniform(r + gap, 1.0 - r - gap) for _ in range(3)]
        ok = True
        for (x, y, z, rr) in out:
            dd = (c[0] - x) ** 2 + (c[1] - y) ** 2 + (c[2] - z) ** 2
            if dd < (r + rr + gap) ** 2:
                ok = False
                break
        if ok:
            out.append((c[0], c[1], c[2], r))
    return np.array(out, dtype=np.float64)


def elasticity3d_voids(cells=64, p=4, alpha=1e-6, n_voids=64, seed=0, quad_depth=3):
    """3D linear elasticity (E=1, nu=0.3) on the unit block perforated by 64
    seed-placed spherical voids of radius 0.03-0.08; clamped face x=0 by
    penalty, unit traction (1,0,0) on the face x=1; traction-free voids."""
    voids = draw_voids(n_voids, seed=seed, gap=1.0 / cells)
    return _base(3, (cells,) * 3, p, pde="elasticity", E=1.0, nu=0.3, alpha=alpha,
                 beta=1e4, geometry=dict(kind="voids", balls=voids.tolist()),
                 source=dict(kind="const", f0=0.0),
                 dirichlet=dict(kind="faces", g="zero", faces=[0]),
                 traction=dict(face=1, t=(1.0, 0.0, 0.0)), quad_depth=quad_depth,
                 name=f"elasticity3d_voids_{cells}^3_p{p}")


def elasticity_mms(dim=3, cells=4, p=2, E=1.0, nu=0.3, beta=1e9, v=(1.0, -2.0, 3.0)):
    """Body-fitted linear elasticity on the unit box (no immersed boundary)
    with the manufactured displacement u = prod_a sin(pi x_a) v: the body force
    that makes it exact and homogeneous Dirichlet data on every face by
    penalty (plane strain in 2D)."""
    return _base(dim, (cells,) * dim, p, pde="elasticity", E=E, nu=nu, alpha=1.0, beta=beta,
                 geometry=dict(kind="none"), source=dict(kind="elastic_sin3", v=tuple(v)),
                 dirichlet=dict(kind="faces", g="zero", faces=list(range(2 * dim))),
                 traction=None, quad_depth=0, name=f"elasticity_mms_{dim}d_{cells}_p{p}")


def poisson3d_sphere_mlhp(cells=16, p=2, overlay_levels=3, alpha=1e-8, radius=0.3,
                          quad_depth=3):
    """The sphere problem of poisson3d_sphere (manufactured sin solution,
    Dirichlet data on the sphere by penalty) with r = 0.3 on a 16^3 base grid
    whose cut cells are overlaid to depth 3 (multi-level hp)."""
    d = poisson3d_sphere(cells=cells, p=p, alpha=alpha, radius=radius, quad_depth=quad_depth)
    d.update(overlay_levels=overlay_levels, smoother="patchwise",
             name=f"poisson3d_sphere_mlhp_{cells}^3_p{p}_k{overlay_levels}")
    return d


def perforated_plate(cells=8, p=2, overlay_levels=0, alpha=1e-8, quad_depth=3):
    """Plane-strain plate [0,4]^2 with four circular cavities of radius
    0.3 sqrt(2) centred in its quadrants, E = 2.069e5, nu = 0.29, clamped on
    x = 0 and pulled by a unit traction on x = 4 (penalty beta = 1e8);
    cut cells overlaid to depth `overlay_levels`.  cells = 8 per axis is the
    mesh size h = 1/8 of the plate side."""
    r = 0.3 * math.sqrt(2.0)
    balls = [(1.0, 1.0, 0.0, r), (3.0, 1.0, 0.0, r), (1.0, 3.0, 0.0, r), (3.0, 3.0, 0.0, r)]
    return _base(2, (cells, cells), p, pde="elasticity", E=2.069e5, nu=0.29, alpha=alpha,
                 beta=1e8, lo=(0.0, 0.0), hi=(4.0, 4.0),
                 geometry=dict(kind="voids", balls=balls), source=dict(kind="const", f0=0.0),
                 dirichlet=dict(kind="faces", g="zero", faces=[0]),
                 traction=dict(face=1, t=(1.0, 0.0, 0.0)), quad_depth=quad_depth,
                 overlay_levels=overlay_levels, smoother="patchwise",
                 name=f"perforated_plate_{cells}^2_p{p}_k{overlay_levels}")


def popcorn_centers(r0=0.6):
    """The twelve bump centres of the popcorn surface (Sec. 4.3.2) on the
    sphere of radius r0: (r0/sqrt 5)(2 cos t_k, 2 sin t_k, +-1) with
    t_k = 2 k pi / 5 (z = +1) and (2k - 1) pi / 5 (z = -1), k = 0..4, and the
    poles (0, 0, +-r0)."""
    s = r0 / math.sqrt(5.0)
    out = []
    for k in range(5):
        t = 2.0 * k * math.pi / 5.0
        out.append((s * 2.0 * math.cos(t), s * 2.0 * math.sin(t), s))
    for k in range(5):
        t = (2.0 * k - 1.0) * math.pi / 5.0
        out.append((s * 2.0 * math.cos(t), s * 2.0 * math.sin(t), -s))
    out += [(0.0, 0.0, r0), (0.0, 0.0, -r0)]
    return out


def popcorn(cells=97, p=3, alpha=1e-6, quad_depth=3, space="trunk", drop_outside=True):
    """Popcorn benchmark (Sec. 4.3.2): the embedding cube (-1, 1)^3, the
    popcorn level set with r0 = 0.6, A = 3, sigma = 0.2, manufactured
    u = x^3 + x y^2 + y^3 + z^4 + sin(3 (x^2 + y^2)) (source -Lap u, Dirichlet
    u on the surface by penalty, beta = 1e4), trunk-space elements, fully
    fictitious cells removed; 97^3 cells, p = 3 is the paper's coarsest mesh."""
    return _base(3, (cells,) * 3, p, lo=(-1.0,) * 3, hi=(1.0,) * 3, alpha=alpha, beta=1e4,
                 geometry=dict(kind="popcorn", r0=0.6, A=3.0, sigma=0.2,
                               centers=popcorn_centers(0.6)),
                 source=dict(kind="popcorn"), dirichlet=dict(kind="levelset", g="popcorn"),
                 quad_depth=quad_depth, space=space, drop_outside=drop_outside,
                 name=f"popcorn_{cells}^3_p{p}")


def cube_cavities(cells=32, p=2, overlay_levels=0, alpha=1e-8, quad_depth=3):
    """Cube with spherical cavities (Sec. 4.3): the perforated plate in 3D, a
    cube of side 4 with eight cavities of radius 0.3 sqrt(2) centred in its
    octants, E = 2.069e5, nu = 0.29, alpha = 1e-8, beta = 1e10, clamped on
    z = 0 and loaded by the pressure 100 on z = 4; trunk-space elements,
    fully fictitious cells removed; h = 4 / cells (32 cells: h = 1/32 of
    the side)."""
    r = 0.3 * math.sqrt(2.0)
    balls = [(x, y, z, r) for z in (1.0, 3.0) for y in (1.0, 3.0) for x in (1.0, 3.0)]
    return _base(3, (cells,) * 3, p, pde="elasticity", E=2.069e5, nu=0.29, alpha=alpha,
                 beta=1e10, lo=(0.0,) * 3, hi=(4.0,) * 3,
                 geometry=dict(kind="voids", balls=balls), source=dict(kind="const", f0=0.0),
                 dirichlet=dict(kind="faces", g="zero", faces=[4]),
                 traction=dict(face=5, t=(0.0, 0.0, -100.0)), quad_depth=quad_depth,
                 overlay_levels=overlay_levels, space="trunk", drop_outside=True,
                 smoother="elementwise" if overlay_levels == 0 else "patchwise",
                 name=f"cube_cavities_{cells}^3_p{p}_k{overlay_levels}")


def random_rotation(rng: SplitMix64) -> list[list[float]]:
    """Rotation matrix of a uniform random unit quaternion (Shoemake 1992)."""
    u1, u2, u3 = rng.uniform(), rng.uniform(), rng.uniform()
    a = math.sqrt(1.0 - u1)
    b = math.sqrt(u1)
    qw = a * math.sin(2 * math.pi * u2)
    qx = a * math.cos(2 * math.pi * u2)
    qy = b * math.sin(2 * math.pi * u3)
    qz = b * math.cos(2 * math.pi * u3)
    return [[1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qz * qw), 2 * (qx * qz + qy * qw)],
            [2 * (qx * qy + qz * qw), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qx * qw)],
            [2 * (qx * qz - qy * qw), 2 * (qy * qz + qx * qw), 1 - 2 * (qx * qx + qy * qy)]]


def batch_instance(i: int, base_seed: int = 0, cmin=8, cmax=32, ps=(2, 3, 4)):
    """Instance i of the batch of independent 3D Poisson problems: C in
    U{8..32}, p in {2,3,4}, an ellipsoid with semi-axes U[0.2,0.45] and a
    uniform random rotation centred in the unit cube, f = 1, homogeneous
    Dirichlet on the ellipsoid surface, alpha = 1e-8."""
    rng = SplitMix64(instance_seed(base_seed, i))
    c = rng.randint(cmin, cmax)
    p = ps[rng.randint(0, len(ps) - 1)]
    axes = [rng.uniform(0.2, 0.45) for _ in range(3)]
    rot = random_rotation(rng)
    return _base(3, (c, c, c), p, alpha=1e-8, beta=1e4,
                 geometry=dict(kind="ellipsoid", center=(0.5, 0.5, 0.5), axes=axes, rot=rot),
                 source=dict(kind="const", f0=1.0),
                 dirichlet=dict(kind="levelset", g="zero"), quad_depth=3,
                 name=f"batch_{base_seed}_{i}_C{c}_p{p}")


def batch(n=256, base_seed=0, **kw):
    return [batch_instance(i, base_seed, **kw) for i in range(n)]


def random_vector(n: int, seed: int = 1) -> np.ndarray:
    """Test vector with entries U(-1, 1), seeded."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=n)


CONFIGS = {
    "poisson2d_circle": poisson2d_circle,
    "poisson3d_sphere": poisson3d_sphere,
    "elasticity3d_voids": elasticity3d_voids,
    "square_mms": square_mms,
    "poisson3d_sphere_mlhp": poisson3d_sphere_mlhp,
    "perforated_plate": perforated_plate,
    "popcorn": popcorn,
    "rotated_square": rotated_square,
    "cube_cavities": cube_cavities,
}
