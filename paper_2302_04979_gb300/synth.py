"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

Holds none of the method's arithmetic: only counter-based random numbers
(splitmix64, Steele, Lea & Flood 2014) and the input recipes of the
benchmark configurations (material fields, source waveform).  The oracle and
the CUDA path receive the same arrays from here.
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, n, stream=0):
    """n outputs of splitmix64 with state seed + (stream << 40) advanced by the golden gamma per draw."""
    with np.errstate(over="ignore"):
        base = np.uint64(seed) + (np.uint64(stream) << np.uint64(40)) * _GOLDEN
        z = base + np.arange(1, n + 1, dtype=np.uint64) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed, n, lo=0.0, hi=1.0, stream=0):
    u = (splitmix64(seed, n, stream) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


def normal(seed, n, stream=0):
    """Standard normals by Box-Muller from two uniform streams."""
    u1 = uniform(seed, n, stream=2 * stream + 1)
    u2 = uniform(seed, n, stream=2 * stream + 2)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


def block_material(seed, blocks=(8, 8, 8), lo=1.0, hi=9.0):
    """Piecewise-constant material on a block grid: array (b_z, b_y, b_x), uniform in [lo, hi)."""
    bx, by, bz = blocks
    return uniform(seed, bx * by * bz, lo, hi, stream=7).reshape(bz, by, bx)


class GaussianBumps:
    """eps(x) = 1 + 3 (1 - prod_k (1 - a_k exp(-|x - c_k|^2 / (2 s_k^2)))), values in [1, 4).

    8 bumps with centres in [0,1]^3, widths in [0.05, 0.2], amplitudes in [0.5, 1].
    """

    def __init__(self, seed, nbumps=8):
        self.c = uniform(seed, 3 * nbumps, 0.0, 1.0, stream=11).reshape(nbumps, 3)
        self.s = uniform(seed, nbumps, 0.05, 0.2, stream=12)
        self.a = uniform(seed, nbumps, 0.5, 1.0, stream=13)

    def __call__(self, x, y, z):
        x, y, z = np.asarray(x, dtype=np.float64), np.asarray(y, dtype=np.float64), np.asarray(z, dtype=np.float64)
        prod = np.ones(np.broadcast(x, y, z).shape)
        for k in range(len(self.s)):
            r2 = (x - self.c[k, 0]) ** 2 + (y - self.c[k, 1]) ** 2 + (z - self.c[k, 2]) ** 2
            prod = prod * (1.0 - self.a[k] * np.exp(-r2 / (2.0 * self.s[k] ** 2)))
        return 1.0 + 3.0 * (1.0 - prod)


def pulse_centre(seed):
    return uniform(seed, 3, 0.3, 0.7, stream=21)


def pulse_profile(centre, width=0.05):
    """Spatial profile of the current J = z-hat g(x) s(t): a Gaussian of the given width."""
    def J(x, y, z):
        r2 = (x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2
        g = np.exp(-r2 / (2.0 * width ** 2))
        return np.array([0.0 * g, 0.0 * g, g])
    return J


def source_amplitudes(dt, nsteps, f0=1.0, tau=0.25, t0=0.75):
    """s(t_n + dt/2) for the Gaussian-modulated carrier s(t) = sin(2 pi f0 t) exp(-(t - t0)^2 / (2 tau^2))."""
    t = (np.arange(nsteps) + 0.5) * dt
    return np.sin(2.0 * np.pi * f0 * t) * np.exp(-((t - t0) ** 2) / (2.0 * tau ** 2))


def bump_coefficients(seed, comp_shapes, comp=2, width=0.05):
    """A smooth source vector for a field with components of shapes (nx, ny, nz): component
    ``comp`` holds exp(-|x - x0|^2 / (2 width^2)) at the normalised index positions
    ((i + 1/2)/nx, (j + 1/2)/ny, (k + 1/2)/nz), x0 = pulse_centre(seed); the others are zero.
    Components are concatenated, x fastest."""
    x0 = pulse_centre(seed)
    parts = []
    for c, (nx, ny, nz) in enumerate(comp_shapes):
        if c != comp:
            parts.append(np.zeros(nx * ny * nz))
            continue
        z, y, x = np.meshgrid((np.arange(nz) + 0.5) / nz, (np.arange(ny) + 0.5) / ny, (np.arange(nx) + 0.5) / nx,
                              indexing="ij")
        r2 = (x - x0[0]) ** 2 + (y - x0[1]) ** 2 + (z - x0[2]) ** 2
        parts.append(np.exp(-r2 / (2.0 * width ** 2)).reshape(-1))
    return np.concatenate(parts)


class SineBumpMap:
    """The curved configuration's map F_i(x) = x_i + a sin(pi x) sin(pi y) sin(pi z) (maps the unit
    cube onto itself) and its Jacobian J[r, c] = dF_r/dx_c, as an input for a host-callback map."""

    def __init__(self, amplitude=0.05):
        self.a = float(amplitude)

    def __call__(self, x, y, z):
        s = np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
        return x + self.a * s, y + self.a * s, z + self.a * s

    def jacobian(self, x, y, z):
        x, y, z = np.broadcast_arrays(np.asarray(x, dtype=np.float64), y, z)
        g = [np.pi * np.cos(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z),
             np.pi * np.sin(np.pi * x) * np.cos(np.pi * y) * np.sin(np.pi * z),
             np.pi * np.sin(np.pi * x) * np.sin(np.pi * y) * np.cos(np.pi * z)]
        return np.array([[(1.0 if r == c else 0.0) + self.a * g[c] for c in range(3)] for r in range(3)])


class ShearMap:
    """A smooth map of the unit cube onto a sheared, bent, squeezed hexahedral domain (not the cube):
    F = (x + 0.2 y z, y + 0.1 sin(pi x), 0.8 z + 0.1 x y), det J >= 0.73 on [0, 1]^3."""

    def __call__(self, x, y, z):
        return x + 0.2 * y * z, y + 0.1 * np.sin(np.pi * x), 0.8 * z + 0.1 * x * y

    def jacobian(self, x, y, z):
        x, y, z = np.broadcast_arrays(np.asarray(x, dtype=np.float64), y, z)
        one, zero = np.ones_like(x), np.zeros_like(x)
        return np.array([[one, 0.2 * z, 0.2 * y],
                         [0.1 * np.pi * np.cos(np.pi * x), one, zero],
                         [0.1 * y, 0.1 * x, 0.8 * one]])


class QuarterCoaxNURBS:
    """The same quarter coaxial cable as a degree-2 NURBS patch (the paper's description of the
    geometry gives no control points; these are the textbook ones): along y^ the quarter circle as a
    rational quadratic with control points (1, 0), (1, 1), (0, 1) and weights 1, sqrt(2)/2, 1; along
    x^ the radius 1 + (sqrt 2 - 1) x^ (degree 1, unchanged by elevation to 2); along z^ the identity.
    F = (r(x^) C_x(y^), r(x^) C_y(y^), z^): the same domain as ``QuarterCoaxMap`` with a non-uniform
    angular speed."""

    dr = np.sqrt(2.0) - 1.0
    w1 = np.sqrt(0.5)

    def _arc(self, y):
        y = np.asarray(y, dtype=np.float64)
        b0, b1, b2 = (1.0 - y) ** 2, 2.0 * y * (1.0 - y), y * y
        den = b0 + self.w1 * b1 + b2
        cx = (b0 + self.w1 * b1) / den
        cy = (self.w1 * b1 + b2) / den
        # derivatives of the quotients
        d0, d1, d2 = -2.0 * (1.0 - y), 2.0 - 4.0 * y, 2.0 * y
        dden = d0 + self.w1 * d1 + d2
        dcx = ((d0 + self.w1 * d1) - cx * dden) / den
        dcy = ((self.w1 * d1 + d2) - cy * dden) / den
        return cx, cy, dcx, dcy

    def __call__(self, x, y, z):
        r = 1.0 + self.dr * np.asarray(x, dtype=np.float64)
        cx, cy, _, _ = self._arc(y)
        return r * cx, r * cy, np.asarray(z, dtype=np.float64) + 0.0 * r

    def jacobian(self, x, y, z):
        x, y, z = np.broadcast_arrays(np.asarray(x, dtype=np.float64), y, z)
        r = 1.0 + self.dr * x
        cx, cy, dcx, dcy = self._arc(y)
        zero, one = np.zeros_like(x), np.ones_like(x)
        return np.array([[self.dr * cx, r * dcx, zero],
                         [self.dr * cy, r * dcy, zero],
                         [zero, zero, one]])


class QuarterCoaxMap:
    """The quarter coaxial cable {1 < x^2 + y^2 < 2, x, y > 0, 0 < z < 1}: radius r = 1 + (sqrt 2 - 1) x^
    and angle theta = (pi/2) y^ (the exact annular geometry that a degree-2 NURBS patch also
    represents), F = (r cos theta, r sin theta, z^), det J = (pi/2)(sqrt 2 - 1) r > 0."""

    dr = np.sqrt(2.0) - 1.0

    def __call__(self, x, y, z):
        r = 1.0 + self.dr * np.asarray(x, dtype=np.float64)
        t = 0.5 * np.pi * np.asarray(y, dtype=np.float64)
        return r * np.cos(t), r * np.sin(t), np.asarray(z, dtype=np.float64) + 0.0 * r

    def jacobian(self, x, y, z):
        x, y, z = np.broadcast_arrays(np.asarray(x, dtype=np.float64), y, z)
        r = 1.0 + self.dr * x
        t = 0.5 * np.pi * y
        zero, one = np.zeros_like(x), np.ones_like(x)
        return np.array([[self.dr * np.cos(t), -0.5 * np.pi * r * np.sin(t), zero],
                         [self.dr * np.sin(t), 0.5 * np.pi * r * np.cos(t), zero],
                         [zero, zero, one]])
