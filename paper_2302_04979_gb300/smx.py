"""Thin Python binding of the C ABI in include/smx.h (argument marshalling only).

Every computation runs in libsmx.so: the step's operations in its CUDA
kernels, the setup (tables, and the L2 projection of initial data) in its
host C++.  This module converts torch tensors to device pointers and checks
status codes.  If the library is missing it raises: there is no CPU fallback.

Names follow the C ABI: ``create``, ``sizes``, ``curl_primal``, ``curl_dual``,
``hodge_apply``, ``pairing_solve``, ``hodge_star``, ``step``, ``energy``, ``cfl``,
``project``, the reverse-mode calls and the batch.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsmx.so")

# ---- constants mirrored from include/smx.h
OK, EINVAL, EGEOM, EMAT, ECUDA, ENONFINITE, ESTATE, ENOMEM, ESINGULAR, ENOSPACE = 0, -1, -2, -3, -4, -5, -6, -7, -8, -9
ETIMEOUT = -10
MODE_TENSOR, MODE_SIMT, MODE_AUTO = 0, 1, 2
GEOM_IDENTITY, GEOM_SINE_BUMP, GEOM_CALLBACK = 0, 1, 2
MAT_CONST, MAT_BLOCKS, MAT_POINTWISE = 0, 1, 2
FIELD_E, FIELD_B, FIELD_H, FIELD_D = 0, 1, 2, 3

MATERIAL_FN = ctypes.CFUNCTYPE(None, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double), ctypes.c_void_p)


FIELD_FN = MATERIAL_FN  # smx_field_fn: the same C signature, 3 values per point
GEOMETRY_FN = ctypes.CFUNCTYPE(None, ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double), ctypes.c_void_p)


class Material(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("value", ctypes.c_double), ("blocks", ctypes.c_int * 3),
                ("block_values", ctypes.POINTER(ctypes.c_double)), ("fn", MATERIAL_FN),
                ("user", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int * 3), ("nel", ctypes.c_int * 3), ("geometry", ctypes.c_int),
                ("geom_amplitude", ctypes.c_double), ("eps", Material), ("mu", Material),
                ("precision", ctypes.c_int), ("geom_fn", GEOMETRY_FN), ("geom_user", ctypes.c_void_p),
                ("scheme1", ctypes.c_int)]


class SmxError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__("%s failed: %s (%d)" % (what, _lib().smx_strerror(status).decode(), status))


_LIB = None

_SIGS = {
    "smx_create": [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_void_p)],
    "smx_destroy": [ctypes.c_void_p],
    "smx_sizes": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
    "smx_comp_shape": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)],
    "smx_workspace_bytes": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)],
    "smx_bind_workspace": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t],
    "smx_set_stream": [ctypes.c_void_p, ctypes.c_void_p],
    "smx_set_graphs": [ctypes.c_void_p, ctypes.c_int],
    "smx_set_mode_kernel": [ctypes.c_void_p, ctypes.c_int],
    "smx_mode_kernel": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)],
    "smx_project": [ctypes.c_void_p, ctypes.c_int, FIELD_FN, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)],
    "smx_device_status": [ctypes.c_void_p],
    "smx_hodge_star_mixed": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p],
    "smx_receivers_set": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p],
    "smx_receivers_eval": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "smx_receivers_adjoint": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p],
    "smx_set_material_blocks": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p],
    "smx_step_adjoint": [ctypes.c_void_p] * 7 + [ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p],
    "smx_adjoint_terminal": [ctypes.c_void_p] * 5,
    "smx_batch_create": [ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)],
    "smx_batch_destroy": [ctypes.c_void_p],
    "smx_batch_workspace_bytes": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)],
    "smx_batch_bind_workspace": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t],
    "smx_batch_set_state": [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 6 + [ctypes.c_double],
    "smx_batch_step": [ctypes.c_void_p, ctypes.c_int],
    "smx_batch_status": [ctypes.c_void_p],
    "smx_batch_set_wait_limit": [ctypes.c_void_p, ctypes.c_double],
    "smx_batch_set_graphs": [ctypes.c_void_p, ctypes.c_int],
    "smx_batch_autotune": [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
    "smx_curl_primal": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double],
    "smx_curl_dual": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                      ctypes.c_double],
    "smx_hodge_apply": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p],
    "smx_pairing_solve": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p],
    "smx_hodge_star": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p],
    "smx_hodge_star_noalloc": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p],
    "smx_step": [ctypes.c_void_p] + [ctypes.c_void_p] * 6 + [ctypes.c_double, ctypes.c_int],
    "smx_scheme1_star": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                         ctypes.POINTER(ctypes.c_int)],
    "smx_step_scheme1": [ctypes.c_void_p] + [ctypes.c_void_p] * 6 + [ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                                                     ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
    "smx_energy_scheme1": [ctypes.c_void_p] * 5 + [ctypes.POINTER(ctypes.c_double)],
    "smx_cfl_scheme1": [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                        ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_double)],
    "smx_energy": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                   ctypes.POINTER(ctypes.c_double)],
    "smx_cfl": [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                ctypes.POINTER(ctypes.c_double)],
    "smx_factor_matrix": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                          ctypes.c_void_p],
    "smx_hodge_mode": [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
    "smx_step_host": [ctypes.c_void_p] + [ctypes.c_void_p] * 6 + [ctypes.c_double, ctypes.c_int],
    "smx_launch_count": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)],
    "smx_set_timing": [ctypes.c_void_p, ctypes.c_int],
    "smx_kernel_times": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)],
    "smx_kernel_work": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                        ctypes.POINTER(ctypes.c_double)],
}

NCLASS = 28
KERNEL_CLASSES = ("curl_primal", "curl_dual", "hodge_block", "hodge_quad", "solve_x", "solve_y", "solve_z",
                  "reduction", "mass_solve_x", "mass_solve_y", "mass_solve_z",
                  "curl_primal_f32", "curl_dual_f32", "hodge_block_f32", "line_f32_x", "line_f32_y", "line_f32_z",
                  "cast", "hodge_quad_f32", "mass_derivative", "receivers",
                  "line_f64tc_x", "line_f64tc_y", "line_f64tc_z", "line_f32tc_x", "line_f32tc_y", "line_f32tc_z", "residual")


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libsmx.so not built: run __graft_entry__.build() (no CPU fallback exists)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        lib.smx_strerror.argtypes = [ctypes.c_int]
        lib.smx_strerror.restype = ctypes.c_char_p
        _LIB = lib
    return _LIB


def library():
    return _lib()


def _check(st, what):
    if st != OK:
        raise SmxError(st, what)


def _ptr(t):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype.is_floating_point and t.element_size() == 8 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def material(spec):
    """Build an smx_material from a number, ('blocks', array (b_z, b_y, b_x)) or a callable f(x, y, z).

    Returns (Material, keepalive) -- keep the second object alive while the context is created.
    """
    m = Material()
    keep = []
    if callable(spec):
        def cb(n, xyz, out, user):
            pts = np.ctypeslib.as_array(xyz, shape=(n, 3))
            res = np.ctypeslib.as_array(out, shape=(n,))
            res[:] = spec(pts[:, 0], pts[:, 1], pts[:, 2])
        fn = MATERIAL_FN(cb)
        keep.append(fn)
        m.kind, m.fn = MAT_POINTWISE, fn
    elif isinstance(spec, tuple) and spec[0] == "blocks":
        vals = np.ascontiguousarray(spec[1], dtype=np.float64)
        keep.append(vals)
        bz, by, bx = vals.shape
        m.kind = MAT_BLOCKS
        m.blocks[0], m.blocks[1], m.blocks[2] = bx, by, bz
        m.block_values = vals.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    else:
        m.kind, m.value = MAT_CONST, float(spec)
    return m, keep


FP64, MIXED, MIXED_REFINED = 0, 1, 2


def geometry_callback(mapping):
    """smx_geometry_fn for a map object: mapping(X, Y, Z) -> (x, y, z) and mapping.jacobian(X, Y, Z)
    -> J[r, c] = dF_r / dxhat_c (arrays over the points), as the seeded input maps provide."""
    def cb(n, xh, x, jac, user):
        pts = np.ctypeslib.as_array(xh, shape=(n, 3))
        X = np.ctypeslib.as_array(x, shape=(n, 3))
        J = np.ctypeslib.as_array(jac, shape=(n, 3, 3))
        try:
            F = mapping(pts[:, 0], pts[:, 1], pts[:, 2])
            X[:] = np.stack([np.asarray(F[r], dtype=np.float64) * np.ones(n) for r in range(3)], axis=1)
            D = np.asarray(mapping.jacobian(pts[:, 0], pts[:, 1], pts[:, 2]), dtype=np.float64)
            J[:] = np.moveaxis(D * np.ones((3, 3, n)), 2, 0)
        except Exception:  # reported as SMX_EGEOM by the library
            X[:] = np.nan
    return GEOMETRY_FN(cb)


def make_params(p, nel, geometry="identity", amplitude=0.05, eps=1.0, mu=1.0, precision="fp64", scheme1=False):
    """geometry: "identity", "sine_bump" (amplitude) or a map object (see geometry_callback)."""
    P = Params()
    p = np.broadcast_to(np.asarray(p, dtype=int), (3,))
    nel = np.broadcast_to(np.asarray(nel, dtype=int), (3,))
    for a in range(3):
        P.p[a], P.nel[a] = int(p[a]), int(nel[a])
    keep = []
    if isinstance(geometry, str):
        P.geometry = {"identity": GEOM_IDENTITY, "sine_bump": GEOM_SINE_BUMP}[geometry]
    else:
        P.geometry = GEOM_CALLBACK
        P.geom_fn = geometry_callback(geometry)
        keep.append(P.geom_fn)
    P.geom_amplitude = float(amplitude)
    P.eps, k1 = material(eps)
    P.mu, k2 = material(mu)
    P.precision = {"fp64": FP64, "mixed": MIXED, "mixed_refined": MIXED_REFINED}[precision]
    P.scheme1 = 1 if scheme1 else 0
    return P, keep + k1 + k2


class Context:
    """Owns an smx_ctx; the device workspace is a torch tensor bound by ``bind``."""

    def __init__(self, p, nel, geometry="identity", amplitude=0.05, eps=1.0, mu=1.0, precision="fp64",
                 scheme1=False):
        lib = _lib()
        P, keep = make_params(p, nel, geometry, amplitude, eps, mu, precision, scheme1)
        h = ctypes.c_void_p()
        _check(lib.smx_create(ctypes.byref(P), ctypes.byref(h)), "smx_create")
        # a geometry callback is called again by smx_project: keep it alive with the context
        self._geometry_fn = keep[0] if not isinstance(geometry, str) else None
        del keep
        self.h = h
        ne, nh = ctypes.c_int64(), ctypes.c_int64()
        _check(lib.smx_sizes(h, ctypes.byref(ne), ctypes.byref(nh)), "smx_sizes")
        self.N_e, self.N_h = ne.value, nh.value
        self.workspace = None

    def __del__(self):
        if getattr(self, "h", None) is not None and _LIB is not None:
            _LIB.smx_destroy(self.h)
            self.h = None

    def comp_shape(self, field, comp):
        s = (ctypes.c_int64 * 3)()
        _check(_lib().smx_comp_shape(self.h, field, comp, s), "smx_comp_shape")
        return tuple(s)

    def workspace_bytes(self):
        n = ctypes.c_size_t()
        _check(_lib().smx_workspace_bytes(self.h, ctypes.byref(n)), "smx_workspace_bytes")
        return n.value

    def bind(self, device="cuda"):
        import torch
        nbytes = self.workspace_bytes()
        ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        ptr = ws.data_ptr()
        aligned = (ptr + 255) & ~255
        _check(_lib().smx_bind_workspace(self.h, ctypes.c_void_p(aligned), nbytes), "smx_bind_workspace")
        self.workspace = ws
        return self

    def set_stream(self, stream):
        _check(_lib().smx_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)),
               "smx_set_stream")

    def set_graphs(self, on):
        _check(_lib().smx_set_graphs(self.h, 1 if on else 0), "smx_set_graphs")

    def set_mode_kernel(self, which):
        """Line operators of the Hodge stars.  Mixed context: dense products on the "tensor" cores
        (exact four-digit slicing) or on FP32 "simt" cores ("auto", the default, is "simt").  FP64 context:
        dense products on the "tensor" cores by exact digit slicing (lines of at most 80 entries),
        banded LU recurrences on the FP64 "simt" pipe, or "auto" (default): per star the faster
        of the two -- tensor cores for a separable star, recurrences for the pairing sweeps."""
        _check(_lib().smx_set_mode_kernel(self.h, {"tensor": MODE_TENSOR, "simt": MODE_SIMT, "auto": MODE_AUTO}[which]),
               "smx_set_mode_kernel")

    def project(self, field, V):
        """L2 projection (host, FP64) of a physical 2-form with vector proxy V(x, y, z) -> (3, n)
        onto the coefficients of FIELD_D (X~^2: d or jhat) or FIELD_B (X^2_{h,0}: b); numpy array."""
        n = self.N_e if field == FIELD_D else self.N_h
        out = np.empty(n, dtype=np.float64)

        def cb(m, xyz, res, _user):
            pts = np.ctypeslib.as_array(xyz, shape=(m, 3))
            r = np.ctypeslib.as_array(res, shape=(m, 3))
            try:
                r[:] = np.asarray(V(pts[:, 0], pts[:, 1], pts[:, 2]), dtype=np.float64).T
            except Exception:  # reported as SMX_ENONFINITE by the library
                r[:] = np.nan

        fn = FIELD_FN(cb)
        _check(_lib().smx_project(self.h, field, fn, None, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "smx_project")
        return out

    def mode_kernel(self):
        """The line-operator kernel the Hodge stars run: "tensor" or "simt"."""
        w = ctypes.c_int()
        _check(_lib().smx_mode_kernel(self.h, ctypes.byref(w)), "smx_mode_kernel")
        return {MODE_TENSOR: "tensor", MODE_SIMT: "simt", MODE_AUTO: "auto"}[w.value]

    def device_status(self):
        """Synchronise; raise SmxError(ETIMEOUT) if a bounded device-side wait gave up since the last call."""
        _check(_lib().smx_device_status(self.h), "smx_device_status")

    def factor_matrix(self, axis, which):
        n = ctypes.c_int64()
        _check(_lib().smx_factor_matrix(self.h, axis, which, ctypes.byref(n), None), "smx_factor_matrix")
        out = np.zeros((n.value, n.value))
        _check(_lib().smx_factor_matrix(self.h, axis, which, ctypes.byref(n), out.ctypes.data_as(ctypes.c_void_p)),
               "smx_factor_matrix")
        return out

    def hodge_mode(self, field):
        m = ctypes.c_int()
        _check(_lib().smx_hodge_mode(self.h, field, ctypes.byref(m)), "smx_hodge_mode")
        return m.value

    # ---- hot-path stages
    def curl_primal(self, e, b, alpha):
        _check(_lib().smx_curl_primal(self.h, _ptr(e), _ptr(b), float(alpha)), "smx_curl_primal")

    def curl_dual(self, h, d, alpha, jhat=None, s=0.0):
        _check(_lib().smx_curl_dual(self.h, _ptr(h), _ptr(d), float(alpha), _ptr(jhat), float(s)), "smx_curl_dual")

    def hodge_apply(self, field, x, y):
        _check(_lib().smx_hodge_apply(self.h, field, _ptr(x), _ptr(y)), "smx_hodge_apply")

    def pairing_solve(self, which, y, x):
        _check(_lib().smx_pairing_solve(self.h, which, _ptr(y), _ptr(x)), "smx_pairing_solve")

    def hodge_star(self, field, x, out):
        _check(_lib().smx_hodge_star(self.h, field, _ptr(x), _ptr(out)), "smx_hodge_star")

    def hodge_star_mixed(self, field, x, out):
        """The mixed step's FP32 Hodge star on its own (context created with precision="mixed")."""
        _check(_lib().smx_hodge_star_mixed(self.h, field, _ptr(x), _ptr(out)), "smx_hodge_star_mixed")

    # ---- reverse mode
    def receivers_set(self, xhat):
        """Receiver points (n x 3 parametric coordinates); before bind()."""
        xh = np.ascontiguousarray(xhat, dtype=np.float64).reshape(-1, 3)
        _check(_lib().smx_receivers_set(self.h, xh.shape[0], xh.ctypes.data_as(ctypes.c_void_p)), "smx_receivers_set")
        self.n_receivers = xh.shape[0]

    def receivers_eval(self, e, out):
        _check(_lib().smx_receivers_eval(self.h, _ptr(e), _ptr(out)), "smx_receivers_eval")

    def receivers_adjoint(self, w, alpha, ebar):
        _check(_lib().smx_receivers_adjoint(self.h, _ptr(w), float(alpha), _ptr(ebar)), "smx_receivers_adjoint")

    def set_material_blocks(self, values):
        """New permittivity block values, array (b_z, b_y, b_x) (the context's block grid)."""
        v = np.ascontiguousarray(values, dtype=np.float64)
        _check(_lib().smx_set_material_blocks(self.h, FIELD_D, v.ctypes.data_as(ctypes.c_void_p)),
               "smx_set_material_blocks")

    def step_adjoint(self, d_n, d_np1, dbar, bbar, dt, ebar=None, jhat=None, amp_bar=None, eps_bar=None):
        _check(_lib().smx_step_adjoint(self.h, _ptr(d_n), _ptr(d_np1), _ptr(dbar), _ptr(bbar), _ptr(ebar), _ptr(jhat),
                                       float(dt), _ptr(amp_bar), _ptr(eps_bar)), "smx_step_adjoint")

    def adjoint_terminal(self, d_N, ebar, dbar, eps_bar=None):
        _check(_lib().smx_adjoint_terminal(self.h, _ptr(d_N), _ptr(ebar), _ptr(dbar), _ptr(eps_bar)),
               "smx_adjoint_terminal")

    def hodge_star_noalloc(self, field, x, out):
        """hodge_star without a bound workspace: tables and scratch in the library's fixed device array."""
        _check(_lib().smx_hodge_star_noalloc(self.h, field, _ptr(x), _ptr(out)), "smx_hodge_star_noalloc")

    def step(self, d, b, e, h, dt, nsteps, jhat=None, amp=None):
        _check(_lib().smx_step(self.h, _ptr(d), _ptr(b), _ptr(e), _ptr(h), _ptr(jhat), _ptr(amp), float(dt),
                               int(nsteps)), "smx_step")

    # ---- scheme 1 (mass-matrix Hodge stars), context created with scheme1=True
    def scheme1_star(self, field, x, out, tol=1e-13, maxit=200):
        it = ctypes.c_int()
        _check(_lib().smx_scheme1_star(self.h, field, _ptr(x), _ptr(out), float(tol), int(maxit), ctypes.byref(it)),
               "smx_scheme1_star")
        return it.value

    def step_scheme1(self, d, b, e, h, dt, nsteps, jhat=None, amp=None, tol=1e-13, maxit=200):
        it = ctypes.c_int()
        _check(_lib().smx_step_scheme1(self.h, _ptr(d), _ptr(b), _ptr(e), _ptr(h), _ptr(jhat), _ptr(amp), float(dt),
                                       int(nsteps), float(tol), int(maxit), ctypes.byref(it)), "smx_step_scheme1")
        return it.value

    def energy_scheme1(self, d, b, e, h):
        out = ctypes.c_double()
        _check(_lib().smx_energy_scheme1(self.h, _ptr(d), _ptr(b), _ptr(e), _ptr(h), ctypes.byref(out)),
               "smx_energy_scheme1")
        return out.value

    def cfl_scheme1(self, iters=300, tol=1e-10, cg_tol=1e-12, cg_maxit=200):
        import torch
        dev = self.workspace.device
        v = torch.empty(self.N_e, dtype=torch.float64, device=dev)
        w = torch.empty_like(v)
        t = torch.empty(self.N_h, dtype=torch.float64, device=dev)
        out = ctypes.c_double()
        _check(_lib().smx_cfl_scheme1(self.h, int(iters), float(tol), _ptr(v), _ptr(w), _ptr(t), float(cg_tol),
                                      int(cg_maxit), ctypes.byref(out)), "smx_cfl_scheme1")
        return out.value

    def step_host(self, d, b, e, h, dt, nsteps, jhat=None, amp=None):
        """Leapfrog on host (CPU, ideally pinned) float64 tensors; copies in and out inside the call."""
        for t in (d, b, e, h):
            if t.is_cuda or t.dtype.itemsize != 8 or not t.is_contiguous():
                raise ValueError("expected contiguous float64 host tensors")
        _check(_lib().smx_step_host(self.h, *[ctypes.c_void_p(t.data_ptr()) for t in (d, b, e, h)], _ptr(jhat),
                                    _ptr(amp), float(dt), int(nsteps)), "smx_step_host")

    def launch_count(self):
        n = ctypes.c_int64()
        _check(_lib().smx_launch_count(self.h, ctypes.byref(n)), "smx_launch_count")
        return n.value

    def set_timing(self, on):
        _check(_lib().smx_set_timing(self.h, 1 if on else 0), "smx_set_timing")

    def kernel_times(self):
        """{class: (milliseconds, launches)} of the launches bracketed since timing was switched on."""
        ms = (ctypes.c_double * NCLASS)()
        cnt = (ctypes.c_int64 * NCLASS)()
        _check(_lib().smx_kernel_times(self.h, ms, cnt), "smx_kernel_times")
        return {KERNEL_CLASSES[k]: (ms[k], cnt[k]) for k in range(NCLASS)}

    def kernel_work(self, cls, field):
        """(FP64 flops, minimal bytes) of one launch of kernel class cls writing field."""
        f, b = ctypes.c_double(), ctypes.c_double()
        _check(_lib().smx_kernel_work(self.h, KERNEL_CLASSES.index(cls) if isinstance(cls, str) else cls, field,
                                      ctypes.byref(f), ctypes.byref(b)), "smx_kernel_work")
        return f.value, b.value

    def energy(self, d, b, e=None, dt=0.0):
        out = (ctypes.c_double * 2)()
        _check(_lib().smx_energy(self.h, _ptr(d), _ptr(b), _ptr(e), float(dt), out), "smx_energy")
        return out[0], out[1]

    def cfl(self, iters=500, tol=1e-12):
        import torch
        dev = self.workspace.device
        v = torch.empty(self.N_e, dtype=torch.float64, device=dev)
        w = torch.empty_like(v)
        t = torch.empty(self.N_h, dtype=torch.float64, device=dev)
        out = ctypes.c_double()
        _check(_lib().smx_cfl(self.h, int(iters), float(tol), _ptr(v), _ptr(w), _ptr(t), ctypes.byref(out)),
               "smx_cfl")
        return out.value


class Batch:
    """Independent cavities (bound contexts, all FP64 or all refined mixed; any map and material)
    stepped by one persistent launch per step, replayed as a CUDA graph on a non-default stream."""

    def __init__(self, contexts, device="cuda"):
        import torch
        self.contexts = list(contexts)
        arr = (ctypes.c_void_p * len(self.contexts))(*[c.h.value for c in self.contexts])
        h = ctypes.c_void_p()
        _check(_lib().smx_batch_create(len(self.contexts), arr, ctypes.byref(h)), "smx_batch_create")
        self.h = h
        n = ctypes.c_size_t()
        _check(_lib().smx_batch_workspace_bytes(h, ctypes.byref(n)), "smx_batch_workspace_bytes")
        ws = torch.empty(n.value + 256, dtype=torch.uint8, device=device)
        aligned = (ws.data_ptr() + 255) & ~255
        _check(_lib().smx_batch_bind_workspace(h, ctypes.c_void_p(aligned), n.value), "smx_batch_bind_workspace")
        self.workspace = ws

    def __del__(self):
        if getattr(self, "h", None) is not None and _LIB is not None:
            _LIB.smx_batch_destroy(self.h)
            self.h = None

    def set_state(self, i, d, b, e, h, dt, jhat=None, amp=None):
        _check(_lib().smx_batch_set_state(self.h, int(i), _ptr(d), _ptr(b), _ptr(e), _ptr(h), _ptr(jhat), _ptr(amp),
                                          float(dt)), "smx_batch_set_state")

    def step(self, nsteps):
        _check(_lib().smx_batch_step(self.h, int(nsteps)), "smx_batch_step")

    def status(self):
        _check(_lib().smx_batch_status(self.h), "smx_batch_status")

    def set_graphs(self, on):
        _check(_lib().smx_batch_set_graphs(self.h, 1 if on else 0), "smx_batch_set_graphs")

    def set_wait_limit(self, seconds):
        """Limit of each grid-barrier wait (seconds; 0 makes every pending wait give up at once)."""
        _check(_lib().smx_batch_set_wait_limit(self.h, float(seconds)), "smx_batch_set_wait_limit")

    def autotune(self, steps=3):
        lw = ctypes.c_int()
        _check(_lib().smx_batch_autotune(self.h, int(steps), ctypes.byref(lw)), "smx_batch_autotune")
        return lw.value
