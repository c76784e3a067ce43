"""Thin Python binding of the nh C ABI (include/nh.h).

Argument marshalling only: every call goes straight to libnh.so and every
step of the computation runs in its CUDA kernels.  Function names match the
C entry points; each takes the context first (for error text) where the C
call does not.  Vectors are torch CUDA tensors (or raw device addresses as
ints); host arrays are numpy arrays.  A missing or unloadable libnh.so raises
ImportError -- there is no fallback path.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnh.so")

NH_OK, NH_ERR_ARG, NH_ERR_CUDA, NH_ERR_OOM, NH_ERR_INVERTED = 0, 1, 2, 3, 4
NH_ERR_NOT_CONVERGED, NH_ERR_NAN, NH_ERR_TIMEOUT, NH_ERR_STATE, NH_ERR_UNSUPPORTED = 5, 6, 7, 8, 9
STATUS_NAMES = {0: "NH_OK", 1: "NH_ERR_ARG", 2: "NH_ERR_CUDA", 3: "NH_ERR_OOM", 4: "NH_ERR_INVERTED",
                5: "NH_ERR_NOT_CONVERGED", 6: "NH_ERR_NAN", 7: "NH_ERR_TIMEOUT", 8: "NH_ERR_STATE",
                9: "NH_ERR_UNSUPPORTED"}
NH_F64, NH_F32, NH_F64X = 0, 1, 2
NH_LAYOUT_CURRENT, NH_LAYOUT_INITIAL, NH_LAYOUT_TAPE = 0, 1, 2

_vp = C.c_void_p
_i64 = C.c_int64
_st = C.c_int

# name -> (restype, argtypes); every symbol here is declared in include/nh.h
SIGNATURES = {
    "nh_create": (_st, [C.POINTER(_vp), C.c_int, _vp]),
    "nh_destroy": (_st, [_vp]),
    "nh_last_error": (C.c_char_p, [_vp]),
    "nh_sync": (_st, [_vp]),
    "nh_launch_count": (_i64, [_vp]),
    "nh_space_box": (_st, [_vp, C.c_int, C.c_int, C.c_int, _vp, C.c_int, C.c_int, C.POINTER(_vp),
                           C.POINTER(_i64), C.POINTER(_i64)]),
    "nh_op_assemble_q1": (_st, [_vp, C.POINTER(C.c_int64), _vp, _vp, _vp]),
    "nh_hex_mesh_numbering": (_st, [C.c_int64, _vp, C.c_int64, _vp, C.c_int, C.POINTER(C.c_int64), _vp, _vp,
                                    C.c_char_p, C.c_int64]),
    "nh_hex_morton_order": (_st, [C.c_int64, _vp, C.c_int64, _vp, _vp]),
    "nh_q1_block_pattern": (_st, [C.c_int64, C.c_int64, _vp, C.POINTER(C.c_int64), _vp, _vp]),
    "nh_space_hex": (_st, [_vp, C.c_int64, _vp, C.c_int64, _vp, C.c_int, C.c_int, C.POINTER(_vp),
                           C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "nh_space_coords": (_st, [_vp, _vp]),
    "nh_space_set_dirichlet": (_st, [_vp, _vp]),
    "nh_space_destroy": (_st, [_vp]),
    "nh_op_create": (_st, [_vp, C.c_double, _vp, C.c_double, C.c_int, C.POINTER(_vp)]),
    "nh_op_level": (_st, [_vp, _vp, C.POINTER(_vp)]),
    "nh_op_destroy": (_st, [_vp]),
    "nh_op_info": (_st, [_vp, C.c_int, C.POINTER(C.c_int), C.POINTER(_i64)]),
    "nh_qdata_setup": (_st, [_vp, _vp, C.POINTER(C.c_double)]),
    "nh_debug_wait_timeout": (_st, [_vp, C.c_int]),
    "nh_op_rediscretize": (_st, [_vp, _vp, C.POINTER(_vp)]),
    "nh_qdata_setup_rediscretized": (_st, [_vp, _vp, _vp, C.POINTER(C.c_double)]),
    "nh_residual": (_st, [_vp, _vp, _vp, _vp]),
    "nh_jacobian_apply": (_st, [_vp, C.c_int, _vp, _vp]),
    "nh_jacobian_apply_host": (_st, [_vp, C.c_int, _vp, _vp]),
    "nh_jacobian_diagonal": (_st, [_vp, C.c_int, _vp]),
    "nh_prolong": (_st, [_vp, _vp, C.c_int, _vp, _vp]),
    "nh_restrict": (_st, [_vp, _vp, C.c_int, _vp, _vp]),
    "nh_dot": (_st, [_vp, _i64, _vp, _vp, C.POINTER(C.c_double)]),
    "nh_profile_enable": (_st, [_vp, C.c_int]),
    "nh_profile_read": (_st, [_vp, C.POINTER(C.c_double), C.POINTER(_i64)]),
    "nh_dot_noalloc": (_st, [_vp, _i64, _vp, _vp, _vp]),
    "nh_mg_default_opts": (_st, [_vp, _vp]),
    "nh_mg_create": (_st, [_vp, _vp, C.POINTER(_vp)]),
    "nh_mg_setup": (_st, [_vp]),
    "nh_mg_level_info": (_st, [_vp, C.c_int, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(C.c_double)]),
    "nh_mg_vcycle": (_st, [_vp, _vp, _vp]),
    "nh_mg_destroy": (_st, [_vp]),
    "nh_linear_solve": (_st, [_vp, _vp, _vp, C.c_double, C.c_int, C.c_int, _vp]),
    "nh_solve": (_st, [_vp, _vp, _vp, _vp]),
    "nh_net_create": (_st, [_vp, C.c_int, C.c_int, _vp, C.c_int, C.c_uint64, C.POINTER(_vp)]),
    "nh_net_destroy": (_st, [_vp]),
    "nh_net_set_tensor_cores": (_st, [_vp, C.c_int]),
    "nh_net_param_count": (_st, [_vp, C.POINTER(_i64)]),
    "nh_net_get_params": (_st, [_vp, _vp]),
    "nh_net_set_params": (_st, [_vp, _vp]),
    "nh_net_forward": (_st, [_vp, _vp, _vp]),
    "nh_net_gradient": (_st, [_vp, _vp, _vp, _vp, C.POINTER(C.c_double)]),
    "nh_net_train_step": (_st, [_vp, C.c_int, _vp, _vp, C.c_float, C.POINTER(C.c_double)]),
    "nh_mg_set_learned": (_st, [_vp, _vp]),
    "nh_mg_collect": (_st, [_vp, _vp, C.c_int, _vp, _vp, C.POINTER(C.c_int)]),
    "nh_fma_peak": (_st, [_vp, C.c_int, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "nh_op_set_scatter": (_st, [_vp, C.c_int]),
}


class MgOpts(C.Structure):
    """Mirror of nh_mg_opts."""
    _fields_ = [("n_levels", C.c_int), ("level_p", C.c_int * 8), ("cheb_degree", C.c_int),
                ("cheb_lo", C.c_double), ("cheb_hi", C.c_double), ("lanczos_iters", C.c_int),
                ("coarse_rtol", C.c_double), ("coarse_maxit", C.c_int), ("coarse_assembled", C.c_int),
                ("mixed", C.c_int), ("seed", C.c_uint64), ("load_steps", C.c_int), ("newton_rtol", C.c_double),
                ("newton_atol", C.c_double), ("newton_maxit", C.c_int), ("krylov_rtol", C.c_double),
                ("krylov_maxit", C.c_int), ("line_search", C.c_int), ("verbose", C.c_int),
                ("learned_accept", C.c_int), ("learned_mode", C.c_int),
                ("fp64_kind", C.c_int), ("coarse_rediscretize", C.c_int), ("nonlinear", C.c_int),
                ("lbfgs_m", C.c_int), ("coarse_solver", C.c_int), ("coarse_fixed", C.c_int),
                ("learned_vectors", C.c_int)]


class SolveReport(C.Structure):
    """Mirror of nh_solve_report."""
    _fields_ = [("status", C.c_int), ("load_steps", C.c_int), ("newton_its", C.c_int), ("krylov_its", C.c_int),
                ("vcycles", C.c_int), ("coarse_its", C.c_int), ("rel_residual", C.c_double),
                ("abs_residual", C.c_double), ("seconds", C.c_double), ("t_setup", C.c_double),
                ("t_krylov", C.c_double), ("t_residual", C.c_double), ("learned_accepted", C.c_int),
                ("learned_rejected", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2204_01722_b300.build`")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


class NhError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _check(st, ctx):
    if st != NH_OK:
        msg = lib.nh_last_error(ctx).decode() if ctx else ""
        raise NhError(st, msg)


def _prec_of(t):
    dt = str(getattr(t, "dtype", ""))
    if dt in ("torch.float64", "float64"):
        return NH_F64
    if dt in ("torch.float32", "float32"):
        return NH_F32
    raise TypeError("vectors must be float64 or float32")


# ---- same-name wrappers ----------------------------------------------------------

def nh_create(device=0, stream=None):
    h = _vp()
    _check(lib.nh_create(C.byref(h), device, stream), None)
    return h.value


def nh_destroy(ctx):
    _check(lib.nh_destroy(ctx), None)


def nh_last_error(ctx):
    return lib.nh_last_error(ctx).decode()


def nh_sync(ctx):
    _check(lib.nh_sync(ctx), ctx)


def nh_debug_wait_timeout(ctx, kind):
    _check(lib.nh_debug_wait_timeout(ctx, int(kind)), ctx)


def nh_launch_count(ctx):
    return int(lib.nh_launch_count(ctx))


def nh_space_box(ctx, nx, ny, nz, vertices, p, q):
    """Returns (space, n_nodes, n_dof)."""
    h = _vp()
    nn, nd = _i64(), _i64()
    V = None if vertices is None else np.ascontiguousarray(vertices, dtype=np.float64)
    _check(lib.nh_space_box(ctx, nx, ny, nz, _ptr(V), p, q, C.byref(h), C.byref(nn), C.byref(nd)), ctx)
    return h.value, nn.value, nd.value


def nh_space_hex(ctx, vertices, hex8, p, q):
    """Unstructured hexahedral mesh; vertices [nv, 3], hex8 [ne, 8] in tensor
    corner order.  Returns (space, n_nodes, n_dof)."""
    h = _vp()
    nn, nd = _i64(), _i64()
    V = np.ascontiguousarray(vertices, dtype=np.float64).reshape(-1, 3)
    H = np.ascontiguousarray(hex8, dtype=np.int64).reshape(-1, 8)
    _check(lib.nh_space_hex(ctx, V.shape[0], _ptr(V), H.shape[0], _ptr(H), p, q, C.byref(h), C.byref(nn),
                            C.byref(nd)), ctx)
    return h.value, nn.value, nd.value


def nh_op_assemble_q1(ctx, op, n_nodes):
    """Assembled Q1 operator: (rowptr [n_nodes + 1], col [nnzb], val [nnzb, 3, 3])."""
    nb = C.c_int64()
    _check(lib.nh_op_assemble_q1(op, C.byref(nb), None, None, None), ctx)
    rp = np.empty(n_nodes + 1, dtype=np.int64)
    cl = np.empty(nb.value, dtype=np.int32)
    val = np.empty((nb.value, 3, 3))
    _check(lib.nh_op_assemble_q1(op, C.byref(nb), _ptr(rp), _ptr(cl), _ptr(val)), ctx)
    return rp, cl, val


def nh_hex_mesh_numbering(vertices, hex8, p):
    """Host-only numbering of nh_space_hex: (emap [ne, (p+1)^3] int32, coords [n_nodes, 3]).
    Raises NhError with the reason on an invalid mesh."""
    V = np.ascontiguousarray(vertices, dtype=np.float64).reshape(-1, 3)
    H = np.ascontiguousarray(hex8, dtype=np.int64).reshape(-1, 8)
    nn = C.c_int64()
    err = C.create_string_buffer(512)
    st = lib.nh_hex_mesh_numbering(V.shape[0], _ptr(V), H.shape[0], _ptr(H), p, C.byref(nn), None, None, err, 512)
    if st != NH_OK:
        raise NhError(st, err.value.decode())
    emap = np.empty((H.shape[0], (p + 1) ** 3), dtype=np.int32)
    X = np.empty((nn.value, 3))
    st = lib.nh_hex_mesh_numbering(V.shape[0], _ptr(V), H.shape[0], _ptr(H), p, C.byref(nn), _ptr(emap), _ptr(X),
                                   err, 512)
    if st != NH_OK:
        raise NhError(st, err.value.decode())
    return emap, X


def nh_hex_morton_order(vertices, hex8):
    """Host-only Z-order of the elements by centroid: perm with hex8[perm] the reordered mesh."""
    V = np.ascontiguousarray(vertices, dtype=np.float64).reshape(-1, 3)
    H = np.ascontiguousarray(hex8, dtype=np.int64).reshape(-1, 8)
    perm = np.empty(H.shape[0], dtype=np.int64)
    st = lib.nh_hex_morton_order(V.shape[0], _ptr(V), H.shape[0], _ptr(H), _ptr(perm))
    if st != NH_OK:
        raise NhError(st, "nh_hex_morton_order: invalid mesh")
    return perm


def nh_q1_block_pattern(emap, n_nodes):
    """Host-only block-row pattern of the Q1 COO assembly: (rowptr [n_nodes + 1], col [nnzb])."""
    E = np.ascontiguousarray(emap, dtype=np.int32).reshape(-1, 8)
    nb = C.c_int64()
    st = lib.nh_q1_block_pattern(E.shape[0], n_nodes, _ptr(E), C.byref(nb), None, None)
    if st != NH_OK:
        raise NhError(st, "nh_q1_block_pattern: invalid element map")
    rp = np.empty(n_nodes + 1, dtype=np.int64)
    cl = np.empty(nb.value, dtype=np.int32)
    lib.nh_q1_block_pattern(E.shape[0], n_nodes, _ptr(E), C.byref(nb), _ptr(rp), _ptr(cl))
    return rp, cl


def nh_space_coords(ctx, space, n_nodes):
    X = np.empty((n_nodes, 3))
    _check(lib.nh_space_coords(space, _ptr(X)), ctx)
    return X


def nh_space_set_dirichlet(ctx, space, mask):
    m = np.ascontiguousarray(np.asarray(mask).astype(np.uint8))
    _check(lib.nh_space_set_dirichlet(space, _ptr(m)), ctx)


def nh_space_destroy(space):
    lib.nh_space_destroy(space)


def nh_op_create(ctx, space, nu, E_per_elem=None, E=1.0, layout=NH_LAYOUT_CURRENT):
    h = _vp()
    Ee = None if E_per_elem is None else np.ascontiguousarray(E_per_elem, dtype=np.float64)
    _check(lib.nh_op_create(space, nu, _ptr(Ee), E, layout, C.byref(h)), ctx)
    return h.value


def nh_op_level(ctx, fine_op, coarse_space):
    h = _vp()
    _check(lib.nh_op_level(fine_op, coarse_space, C.byref(h)), ctx)
    return h.value


def nh_op_destroy(op):
    lib.nh_op_destroy(op)


def nh_op_info(ctx, op, prec=NH_F64):
    S = C.c_int()
    b = _i64()
    _check(lib.nh_op_info(op, prec, C.byref(S), C.byref(b)), ctx)
    return S.value, b.value


def nh_qdata_setup(ctx, op, u):
    mj = C.c_double()
    _check(lib.nh_qdata_setup(op, _ptr(u), C.byref(mj)), ctx)
    return mj.value


def nh_op_rediscretize(ctx, fine_op, coarse_space):
    h = _vp()
    _check(lib.nh_op_rediscretize(fine_op, coarse_space, C.byref(h)), ctx)
    return h.value


def nh_qdata_setup_rediscretized(ctx, op, fine_op, u_fine):
    mj = C.c_double()
    _check(lib.nh_qdata_setup_rediscretized(op, fine_op, _ptr(u_fine), C.byref(mj)), ctx)
    return mj.value


def nh_residual(ctx, op, u, g_bc, r):
    _check(lib.nh_residual(op, _ptr(u), _ptr(g_bc), _ptr(r)), ctx)


def nh_jacobian_apply(ctx, op, du, y, prec=None):
    prec = _prec_of(du) if prec is None else prec
    _check(lib.nh_jacobian_apply(op, prec, _ptr(du), _ptr(y)), ctx)


def nh_jacobian_apply_host(ctx, op, du_host, y_host, prec=None):
    prec = _prec_of(du_host) if prec is None else prec
    _check(lib.nh_jacobian_apply_host(op, prec, _ptr(du_host), _ptr(y_host)), ctx)


def nh_jacobian_diagonal(ctx, op, diag, prec=None):
    prec = _prec_of(diag) if prec is None else prec
    _check(lib.nh_jacobian_diagonal(op, prec, _ptr(diag)), ctx)


def nh_prolong(ctx, coarse, fine, uc, uf, prec=None):
    prec = _prec_of(uc) if prec is None else prec
    _check(lib.nh_prolong(coarse, fine, prec, _ptr(uc), _ptr(uf)), ctx)


def nh_restrict(ctx, fine, coarse, rf, rc, prec=None):
    prec = _prec_of(rf) if prec is None else prec
    _check(lib.nh_restrict(fine, coarse, prec, _ptr(rf), _ptr(rc)), ctx)


def nh_dot(ctx, n, x, y):
    r = C.c_double()
    _check(lib.nh_dot(ctx, n, _ptr(x), _ptr(y), C.byref(r)), ctx)
    return r.value


def nh_profile_enable(ctx, on=True):
    _check(lib.nh_profile_enable(ctx, 1 if on else 0), ctx)


def nh_profile_read(ctx):
    """Returns (total_ms, launches) of Jacobian-apply kernels since the last read."""
    ms = C.c_double()
    k = _i64()
    _check(lib.nh_profile_read(ctx, C.byref(ms), C.byref(k)), ctx)
    return ms.value, k.value


NH_DOT_NOALLOC_MAX_N = 1 << 28


def nh_dot_noalloc(stream, n, x, y, result):
    """Allocation-free dot product into the device scalar `result` (stream-ordered)."""
    st = lib.nh_dot_noalloc(stream, n, _ptr(x), _ptr(y), _ptr(result))
    if st != NH_OK:
        raise NhError(st, "nh_dot_noalloc")


def nh_op_set_scatter(ctx, op, mode):
    """0 = atomic scatter-add, 1 = eight-colour passes without atomics."""
    _check(lib.nh_op_set_scatter(op, mode), ctx)


def nh_fma_peak(ctx, prec, iters):
    """Measured FMA throughput (TFLOP/s) and the timed launch (ms)."""
    tf, ms = C.c_double(), C.c_double()
    _check(lib.nh_fma_peak(ctx, prec, iters, C.byref(tf), C.byref(ms)), ctx)
    return tf.value, ms.value


def nh_mg_default_opts(ctx, fine_op, **kw):
    """Default options for `fine_op`, with any field overridden by keyword
    (level_p may be given as a sequence)."""
    o = MgOpts()
    _check(lib.nh_mg_default_opts(fine_op, C.byref(o)), ctx)
    for k, v in kw.items():
        if k == "level_p":
            o.n_levels = len(v)
            for i, pv in enumerate(v):
                o.level_p[i] = pv
        else:
            setattr(o, k, v)
    return o


def nh_mg_create(ctx, fine_op, opts=None):
    h = _vp()
    _check(lib.nh_mg_create(fine_op, None if opts is None else C.byref(opts), C.byref(h)), ctx)
    return h.value


def nh_mg_setup(ctx, mg):
    _check(lib.nh_mg_setup(mg), ctx)


def nh_mg_level_info(ctx, mg, level):
    """Returns (space, op, lambda_max)."""
    s, o, lm = _vp(), _vp(), C.c_double()
    _check(lib.nh_mg_level_info(mg, level, C.byref(s), C.byref(o), C.byref(lm)), ctx)
    return s.value, o.value, lm.value


def nh_mg_vcycle(ctx, mg, r, z):
    _check(lib.nh_mg_vcycle(mg, _ptr(r), _ptr(z)), ctx)


def nh_mg_destroy(mg):
    lib.nh_mg_destroy(mg)


def nh_linear_solve(ctx, mg, b, x, rtol=1e-8, maxit=500, norm=1, check=True):
    rep = SolveReport()
    st = lib.nh_linear_solve(mg, _ptr(b), _ptr(x), rtol, maxit, norm, C.byref(rep))
    if check:
        _check(st, ctx)
    return rep


def nh_solve(ctx, mg, g_bc, u, check=True):
    rep = SolveReport()
    st = lib.nh_solve(mg, _ptr(g_bc), _ptr(u), C.byref(rep))
    if check:
        _check(st, ctx)
    return rep


def nh_net_create(ctx, N, levels, channels, bf16=True, seed=0):
    h = _vp()
    ch = np.ascontiguousarray(channels, dtype=np.int32)
    _check(lib.nh_net_create(ctx, N, levels, _ptr(ch), 1 if bf16 else 0, seed, C.byref(h)), ctx)
    return h.value


def nh_net_destroy(net):
    lib.nh_net_destroy(net)


def nh_net_set_tensor_cores(ctx, net, on):
    _check(lib.nh_net_set_tensor_cores(net, 1 if on else 0), ctx)


def nh_net_param_count(ctx, net):
    k = _i64()
    _check(lib.nh_net_param_count(net, C.byref(k)), ctx)
    return k.value


def nh_net_get_params(ctx, net):
    th = np.empty(nh_net_param_count(ctx, net), dtype=np.float32)
    _check(lib.nh_net_get_params(net, _ptr(th)), ctx)
    return th


def nh_net_set_params(ctx, net, theta):
    th = np.ascontiguousarray(theta, dtype=np.float32)
    _check(lib.nh_net_set_params(net, _ptr(th)), ctx)


def nh_net_forward(ctx, net, x, y):
    _check(lib.nh_net_forward(net, _ptr(x), _ptr(y)), ctx)


def nh_net_gradient(ctx, net, x, t, dparams):
    loss = C.c_double()
    _check(lib.nh_net_gradient(net, _ptr(x), _ptr(t), _ptr(dparams), C.byref(loss)), ctx)
    return loss.value


def nh_net_train_step(ctx, net, batch, x, t, lr):
    loss = C.c_double()
    _check(lib.nh_net_train_step(net, batch, _ptr(x), _ptr(t), lr, C.byref(loss)), ctx)
    return loss.value


def nh_mg_set_learned(ctx, mg, net):
    _check(lib.nh_mg_set_learned(mg, net), ctx)


def nh_mg_collect(ctx, mg, b, max_pairs, feats, targets):
    k = C.c_int()
    _check(lib.nh_mg_collect(mg, _ptr(b), max_pairs, _ptr(feats), _ptr(targets), C.byref(k)), ctx)
    return k.value
