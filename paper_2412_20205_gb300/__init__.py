"""GB300-native extrapolated geometric multigrid for isogeometric Poisson problems.

Thin Python binding of the C-ABI library ``libigamg.so`` (declared in
``include/igamg.h``).  The functions below carry the C names and only marshal
arguments; every step of the solve runs in the library's CUDA kernels.
PyTorch is used for device memory and streams only.  If the library has not
been built, or no CUDA device is present for a GPU call, the calls raise --
there is no CPU fallback.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libigamg.so")

IGAMG_OK, IGAMG_EINVAL, IGAMG_ENOMEM, IGAMG_ECUDA, IGAMG_ENOTCONV, IGAMG_EBREAKDOWN, IGAMG_ETIMEOUT = range(7)
IGAMG_EXTRAP_NONE, IGAMG_RRE, IGAMG_MPE = 0, 1, 2
IGAMG_FP64, IGAMG_FP32_IR, IGAMG_FP32_IR_LEARNED = 0, 1, 2
IGAMG_FLAG_X0_GIVEN, IGAMG_FLAG_ABS_TOL, IGAMG_FLAG_NO_GRAPH, IGAMG_FLAG_HOST_LOOP = 1, 2, 4, 8
IGAMG_SMOOTH_GS, IGAMG_SMOOTH_JACOBI = 0, 1
SMOOTHER = {"gs": IGAMG_SMOOTH_GS, "jacobi": IGAMG_SMOOTH_JACOBI}

EXTRAP = {"none": IGAMG_EXTRAP_NONE, "rre": IGAMG_RRE, "mpe": IGAMG_MPE}
PREC = {"fp64": IGAMG_FP64, "fp32_ir": IGAMG_FP32_IR, "fp32_ir_learned": IGAMG_FP32_IR_LEARNED}

_lib = None


class IgamgError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        lib = _load()
        super().__init__(f"{where}: {lib.igamg_status_str(status).decode()} "
                         f"({lib.igamg_last_error().decode()})")


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    c_int, c_double, c_long, c_size = ctypes.c_int, ctypes.c_double, ctypes.c_long, ctypes.c_size_t
    vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    sigs = {
        "igamg_setup": (c_int, [c_int, c_int, ip, c_int, ctypes.POINTER(vp)]),
        "igamg_assemble": (c_int, [vp]),
        "igamg_info": (c_int, [vp, ip, ip]),
        "igamg_get_factor": (c_int, [vp, c_int, c_int, c_int, dp, ip, ip]),
        "igamg_workspace_bytes": (c_size, [vp, c_int, c_int]),
        "igamg_rhs_sine": (c_int, [vp, c_int, dp, vp, vp]),
        "igamg_setup_general": (c_int, [c_int, ip, c_int, ctypes.POINTER(vp)]),
        "igamg_quadrature_count": (c_long, [vp]),
        "igamg_quadrature_points": (c_int, [vp, dp, dp]),
        "igamg_assemble_general": (c_int, [vp, dp, dp]),
        "igamg_rhs_points": (c_int, [vp, dp, vp, vp]),
        "igamg_solve": (c_int, [vp, vp, vp, c_double, c_int, c_int, c_int, c_int, ctypes.c_uint,
                                vp, c_size, vp, dp, ip, ip]),
        "igamg_apply": (c_int, [vp, c_int, vp, vp, vp, c_size, vp]),
        "igamg_smooth": (c_int, [vp, c_int, vp, vp, c_int, vp, c_size, vp]),
        "igamg_restrict": (c_int, [vp, c_int, vp, vp, vp, c_size, vp]),
        "igamg_prolong": (c_int, [vp, c_int, vp, vp, vp, c_size, vp]),
        "igamg_coarse_solve": (c_int, [vp, vp, vp, vp]),
        "igamg_vcycle": (c_int, [vp, vp, vp, c_int, vp, c_size, vp]),
        "igamg_extrap_workspace_bytes": (c_size, [c_long, c_int]),
        "igamg_extrapolate": (c_int, [c_long, c_int, c_int, vp, c_long, vp, dp, ip, vp, c_size, vp]),
        "igamg_extrapolate_noalloc": (c_int, [c_long, c_int, c_int, vp, c_long, vp, dp, ip, vp]),
        "igamg_destroy": (None, [vp]),
        "igamg_set_smoother": (c_int, [vp, vp, c_double]),
        "igamg_smoother_fell_back": (c_int, [vp]),
        "igamg_coarse_tail_level": (c_int, [vp]),
        "igamg_set_schedule": (c_int, [vp, c_int, c_int]),
        "igamg_get_schedule": (None, [vp, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
        "igamg_set_tail_ctas": (c_int, [vp, c_int]),
        "igamg_get_tail_ctas": (c_int, [vp]),
        "igamg_tail_levels_available": (c_int, [vp, c_int]),
        "igamg_batch_set_tail_ctas": (c_int, [vp, c_int]),
        "igamg_set_cycle": (c_int, [vp, c_int, c_int, c_double]),
        "igamg_get_cycle": (None, [vp, ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(c_double)]),
        "igamg_set_sweep_form": (c_int, [vp, c_int, c_int]),
        "igamg_get_sweep_form": (None, [vp, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
        "igamg_set_wait_limit": (None, [c_double, c_int]),
        "igamg_device_status": (c_int, [vp, vp, c_size, vp]),
        "igamg_set_launch_overlap": (None, [c_int]),
        "igamg_get_launch_overlap": (c_int, []),
        "igamg_autotune": (c_int, [vp, vp, c_size, vp, c_int]),
        "igamg_batch_autotune": (c_int, [vp, vp, c_size, vp, c_int]),
        "igamg_smooth_f32": (c_int, [vp, c_int, vp, vp, c_int, c_int, vp, c_size, vp]),
        "igamg_set_coarse_tail": (c_int, [vp, c_int]),
        "igamg_vcycle_probe": (c_int, [vp, vp, vp, vp, vp, c_size, vp]),
        "igamg_training_workspace_bytes": (c_size, [vp, c_int]),
        "igamg_training_pairs": (c_int, [vp, vp, vp, c_int, c_double, c_int, vp, vp, c_int, vp, c_size, vp, ip]),
        "igamg_cnn_num_weights": (c_int, []),
        "igamg_cnn_workspace_bytes": (c_size, [c_int, c_int, c_int]),
        "igamg_cnn_forward": (c_int, [c_int, c_int, c_int, vp, vp, vp, vp, c_size, vp]),
        "igamg_cnn_grad": (c_int, [c_int, c_int, c_int, vp, vp, vp, vp, vp, vp, c_size, vp]),
        "igamg_adam_step": (c_int, [c_int, vp, vp, vp, vp, c_int, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_float, ctypes.c_float, vp]),
        "igamg_batch_create": (c_int, [c_int, c_int, ip, ip, ctypes.POINTER(vp)]),
        "igamg_batch_layout": (c_int, [vp, ctypes.POINTER(c_long)]),
        "igamg_batch_workspace_bytes": (c_size, [vp, c_int, c_int]),
        "igamg_batch_rhs_sine": (c_int, [vp, c_int, dp, vp, vp]),
        "igamg_batch_solve": (c_int, [vp, vp, vp, c_double, c_int, c_int, c_int, c_int, vp, c_size, vp,
                                      ip, ip, dp]),
        "igamg_batch_destroy": (None, [vp]),
        "igamg_batch_set_device_loop": (c_int, [vp, c_int]),
        "igamg_status_str": (ctypes.c_char_p, [c_int]),
        "igamg_last_error": (ctypes.c_char_p, []),
        "igamg_launch_count": (ctypes.c_longlong, []),
        "igamg_profile_start": (None, []),
        "igamg_profile_stop": (c_long, [c_int, ctypes.c_char_p, c_int, dp, ip]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def lib():
    """The loaded ctypes library (raises if it has not been built)."""
    return _load()


def _check(status, where):
    if status != IGAMG_OK:
        raise IgamgError(status, where)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dbl(arr):
    return arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ------------------------------------------------------------------ C names
def igamg_setup(dim, p, n_elems, n_levels=0):
    n = list(n_elems) if hasattr(n_elems, "__len__") else [int(n_elems)] * dim
    arr = (ctypes.c_int * 3)(*(n + [1] * (3 - len(n))))
    ctx = ctypes.c_void_p()
    _check(_load().igamg_setup(dim, p, arr, n_levels, ctypes.byref(ctx)), "igamg_setup")
    return ctx


def igamg_assemble(ctx):
    _check(_load().igamg_assemble(ctx), "igamg_assemble")


def igamg_info(ctx):
    nl = ctypes.c_int()
    _check(_load().igamg_info(ctx, ctypes.byref(nl), None), "igamg_info")
    m = (ctypes.c_int * (3 * nl.value))()
    _check(_load().igamg_info(ctx, ctypes.byref(nl), m), "igamg_info")
    return [tuple(m[3 * l:3 * l + 3]) for l in range(nl.value)]


def igamg_get_factor(ctx, level, d, which):
    import numpy as np
    rows, cols = ctypes.c_int(), ctypes.c_int()
    _check(_load().igamg_get_factor(ctx, level, d, which, None, ctypes.byref(rows), ctypes.byref(cols)),
           "igamg_get_factor")
    out = np.zeros((rows.value, cols.value))
    _check(_load().igamg_get_factor(ctx, level, d, which, _dbl(out), ctypes.byref(rows), ctypes.byref(cols)),
           "igamg_get_factor")
    return out


def igamg_workspace_bytes(ctx, k, prec):
    return int(_load().igamg_workspace_bytes(ctx, k, prec))


def igamg_rhs_sine(ctx, coeffs, b, stream=None):
    import numpy as np
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    _check(_load().igamg_rhs_sine(ctx, c.shape[0], _dbl(c), _ptr(b), _stream(stream)), "igamg_rhs_sine")


def igamg_setup_general(p, n_elems, n_levels=0):
    n = list(n_elems) if hasattr(n_elems, "__len__") else [int(n_elems)] * 2
    arr = (ctypes.c_int * 3)(*(n + [1]))
    ctx = ctypes.c_void_p()
    _check(_load().igamg_setup_general(p, arr, n_levels, ctypes.byref(ctx)), "igamg_setup_general")
    return ctx


def igamg_quadrature_points(ctx):
    """(xi, eta) arrays of the finest level's quadrature points (x fastest)."""
    import numpy as np
    nq = int(_load().igamg_quadrature_count(ctx))
    xi, eta = np.zeros(nq), np.zeros(nq)
    _check(_load().igamg_quadrature_points(ctx, _dbl(xi), _dbl(eta)), "igamg_quadrature_points")
    return xi, eta


def igamg_assemble_general(ctx, coef, jac=None):
    """coef: (6, nq) A11, A12, A22, B1, B2, c at the mapped points; jac: (4, nq) or None."""
    import numpy as np
    cf = np.ascontiguousarray(coef, dtype=np.float64)
    jc = None if jac is None else np.ascontiguousarray(jac, dtype=np.float64)
    _check(_load().igamg_assemble_general(ctx, _dbl(cf), None if jc is None else _dbl(jc)),
           "igamg_assemble_general")


def igamg_rhs_points(ctx, f, b, stream=None):
    import numpy as np
    fv = np.ascontiguousarray(f, dtype=np.float64)
    _check(_load().igamg_rhs_points(ctx, _dbl(fv), _ptr(b), _stream(stream)), "igamg_rhs_points")


def igamg_solve(ctx, b, x, tol, extrap, k, max_cycles, prec, flags, ws, stream=None):
    """Returns (status, history[0..cycles], cycles, vcycles); ENOTCONV is not raised."""
    import numpy as np
    hist = np.zeros(max_cycles + 1)
    cyc, vc = ctypes.c_int(), ctypes.c_int()
    st = _load().igamg_solve(ctx, _ptr(b), _ptr(x), tol, extrap, k, max_cycles, prec, flags,
                             _ptr(ws), ws.numel() * ws.element_size(), _stream(stream), _dbl(hist),
                             ctypes.byref(cyc), ctypes.byref(vc))
    if st not in (IGAMG_OK, IGAMG_ENOTCONV):
        _check(st, "igamg_solve")
    return st, hist[: cyc.value + 1], cyc.value, vc.value


def igamg_apply(ctx, level, x, y, ws, stream=None):
    _check(_load().igamg_apply(ctx, level, _ptr(x), _ptr(y), _ptr(ws), ws.numel(), _stream(stream)),
           "igamg_apply")


def igamg_smooth(ctx, level, x, b, descending, ws, stream=None):
    _check(_load().igamg_smooth(ctx, level, _ptr(x), _ptr(b), int(descending), _ptr(ws), ws.numel(),
                                _stream(stream)), "igamg_smooth")


def igamg_restrict(ctx, level, fine, coarse, ws, stream=None):
    _check(_load().igamg_restrict(ctx, level, _ptr(fine), _ptr(coarse), _ptr(ws), ws.numel(),
                                  _stream(stream)), "igamg_restrict")


def igamg_prolong(ctx, level, coarse, fine, ws, stream=None):
    _check(_load().igamg_prolong(ctx, level, _ptr(coarse), _ptr(fine), _ptr(ws), ws.numel(),
                                 _stream(stream)), "igamg_prolong")


def igamg_coarse_solve(ctx, r, e, stream=None):
    _check(_load().igamg_coarse_solve(ctx, _ptr(r), _ptr(e), _stream(stream)), "igamg_coarse_solve")


def igamg_vcycle(ctx, x, b, prec, ws, stream=None):
    _check(_load().igamg_vcycle(ctx, _ptr(x), _ptr(b), prec, _ptr(ws), ws.numel(), _stream(stream)),
           "igamg_vcycle")


def igamg_extrap_workspace_bytes(n, q):
    return int(_load().igamg_extrap_workspace_bytes(n, q))


def igamg_extrapolate(n, q, method, S, ld, t, ws, stream=None):
    import numpy as np
    gamma = np.zeros(q + 2)
    qused = ctypes.c_int()
    _check(_load().igamg_extrapolate(n, q, method, _ptr(S), ld, _ptr(t), _dbl(gamma), ctypes.byref(qused),
                                     _ptr(ws), ws.numel(), _stream(stream)), "igamg_extrapolate")
    return gamma, qused.value


def igamg_extrapolate_noalloc(n, q, method, S, ld, t, stream=None):
    """igamg_extrapolate with the library's built-in scratch (no workspace)."""
    import numpy as np
    gamma = np.zeros(q + 2)
    qused = ctypes.c_int()
    _check(_load().igamg_extrapolate_noalloc(n, q, method, _ptr(S), ld, _ptr(t), _dbl(gamma),
                                             ctypes.byref(qused), _stream(stream)), "igamg_extrapolate_noalloc")
    return gamma, qused.value


def igamg_destroy(ctx):
    _load().igamg_destroy(ctx)


def igamg_launch_count():
    return int(_load().igamg_launch_count())


def igamg_profile_start():
    _load().igamg_profile_start()


def igamg_profile_stop(cap=20000, name_len=96):
    """Per-launch records [(kernel name, microseconds, grid CTAs)] since igamg_profile_start."""
    import numpy as np
    names = ctypes.create_string_buffer(cap * name_len)
    us = np.zeros(cap)
    grid = (ctypes.c_int * cap)()
    n = int(_load().igamg_profile_stop(cap, names, name_len, _dbl(us), grid))
    raw = names.raw
    out = []
    for i in range(min(n, cap)):
        nm = raw[i * name_len:(i + 1) * name_len].split(b"\0", 1)[0].decode(errors="replace")
        out.append((nm, float(us[i]), int(grid[i])))
    return out


def igamg_set_smoother(ctx, w, stall_ratio=0.95):
    _check(_load().igamg_set_smoother(ctx, _ptr(w), stall_ratio), "igamg_set_smoother")


def igamg_smoother_fell_back(ctx):
    return bool(_load().igamg_smoother_fell_back(ctx))


def igamg_smooth_f32(ctx, level, x, b, descending, ws, sums_current=False, stream=None):
    _check(_load().igamg_smooth_f32(ctx, level, _ptr(x), _ptr(b), int(descending), int(bool(sums_current)),
                                    _ptr(ws), ws.numel(), _stream(stream)), "igamg_smooth_f32")


def igamg_set_schedule(ctx, gs_threads=0, tail_levels=-1):
    _check(_load().igamg_set_schedule(ctx, gs_threads, tail_levels), "igamg_set_schedule")


def igamg_set_cycle(ctx, smoother="gs", mu=1, omega=2.0 / 3.0):
    """Cycle of Algorithm 2: smoother 'gs' or 'jacobi' (weight omega), mu = 1 (V) or 2 (W)."""
    _check(_load().igamg_set_cycle(ctx, SMOOTHER[smoother], mu, omega), "igamg_set_cycle")


def igamg_get_cycle(ctx):
    a, b, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _load().igamg_get_cycle(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(w))
    return {"smoother": "jacobi" if a.value == IGAMG_SMOOTH_JACOBI else "gs", "mu": b.value, "omega": w.value}


def igamg_set_sweep_form(ctx, single_launch_fp32=-1, single_launch_fp64=-1):
    """GS sweep form per precision: 1 one launch per sweep, 0 one per row phase, -1 unchanged."""
    _check(_load().igamg_set_sweep_form(ctx, int(single_launch_fp32), int(single_launch_fp64)),
           "igamg_set_sweep_form")


def igamg_get_sweep_form(ctx):
    a, b = ctypes.c_int(), ctypes.c_int()
    _load().igamg_get_sweep_form(ctx, ctypes.byref(a), ctypes.byref(b))
    return {"fp32": a.value, "fp64": b.value}


def igamg_set_wait_limit(seconds=1.0, test_unset_flag=False):
    """Process-wide bound of the device-side waits (test_unset_flag: make them run out)."""
    _load().igamg_set_wait_limit(float(seconds), 1 if test_unset_flag else 0)


def igamg_device_status(ctx, ws, stream=None):
    """IGAMG_OK, or IGAMG_ETIMEOUT if a bounded device wait gave up (returned, not raised)."""
    st = _load().igamg_device_status(ctx, _ptr(ws), ws.numel(), _stream(stream))
    if st not in (IGAMG_OK, IGAMG_ETIMEOUT):
        _check(st, "igamg_device_status")
    return st


def igamg_set_launch_overlap(enable):
    """Process-wide: launch the V-cycle chain with programmatic stream serialisation."""
    _load().igamg_set_launch_overlap(1 if enable else 0)


def igamg_get_launch_overlap():
    return bool(_load().igamg_get_launch_overlap())


def igamg_get_schedule(ctx):
    a, b = ctypes.c_int(), ctypes.c_int()
    _load().igamg_get_schedule(ctx, ctypes.byref(a), ctypes.byref(b))
    return {"gs_threads": a.value, "tail_levels": b.value, "tail_ctas": _load().igamg_get_tail_ctas(ctx)}


def igamg_set_tail_ctas(ctx, ctas):
    """Coarse tail on one CTA (1) or on a thread-block cluster of 8 or 16 CTAs."""
    _check(_load().igamg_set_tail_ctas(ctx, int(ctas)), "igamg_set_tail_ctas")


def igamg_tail_levels_available(ctx, ctas):
    """Deepest tail level of the one-CTA (ctas = 1) or cluster (8, 16) form; 0: none."""
    return _load().igamg_tail_levels_available(ctx, int(ctas))


def igamg_autotune(ctx, ws, reps=3, stream=None):
    _check(_load().igamg_autotune(ctx, _ptr(ws), ws.numel(), _stream(stream), reps), "igamg_autotune")
    return igamg_get_schedule(ctx)


def igamg_batch_autotune(batch, ws, reps=3, stream=None):
    _check(_load().igamg_batch_autotune(batch, _ptr(ws), ws.numel(), _stream(stream), reps),
           "igamg_batch_autotune")


def igamg_coarse_tail_level(ctx):
    return int(_load().igamg_coarse_tail_level(ctx))


def igamg_set_coarse_tail(ctx, enable):
    _check(_load().igamg_set_coarse_tail(ctx, int(bool(enable))), "igamg_set_coarse_tail")


def igamg_vcycle_probe(ctx, x, b, x_mid, ws, stream=None):
    _check(_load().igamg_vcycle_probe(ctx, _ptr(x), _ptr(b), _ptr(x_mid), _ptr(ws), ws.numel(), _stream(stream)),
           "igamg_vcycle_probe")


def igamg_training_workspace_bytes(ctx, k):
    return int(_load().igamg_training_workspace_bytes(ctx, k))


def igamg_training_pairs(ctx, b, uh, k, tol, max_restarts, R, E, ws, stream=None):
    """Writes scaled (r, e) training pairs into the FP32 tensors R, E (pairs x N); returns the count."""
    n = ctypes.c_int()
    max_pairs = min(R.shape[0], E.shape[0])
    _check(_load().igamg_training_pairs(ctx, _ptr(b), _ptr(uh), k, tol, max_restarts, _ptr(R), _ptr(E), max_pairs,
                                        _ptr(ws), ws.numel(), _stream(stream), ctypes.byref(n)),
           "igamg_training_pairs")
    return n.value


def igamg_cnn_num_weights():
    return int(_load().igamg_cnn_num_weights())


def igamg_cnn_workspace_bytes(batch, H, W):
    return int(_load().igamg_cnn_workspace_bytes(batch, H, W))


def igamg_cnn_forward(batch, H, W, r, w, y, ws, stream=None):
    _check(_load().igamg_cnn_forward(batch, H, W, _ptr(r), _ptr(w), _ptr(y), _ptr(ws), ws.numel(),
                                     _stream(stream)), "igamg_cnn_forward")


def igamg_cnn_grad(batch, H, W, r, e, w, grad, loss, ws, stream=None):
    _check(_load().igamg_cnn_grad(batch, H, W, _ptr(r), _ptr(e), _ptr(w), _ptr(grad), _ptr(loss), _ptr(ws),
                                  ws.numel(), _stream(stream)), "igamg_cnn_grad")


def igamg_adam_step(w, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8, stream=None):
    _check(_load().igamg_adam_step(w.numel(), _ptr(w), _ptr(g), _ptr(m), _ptr(v), step, lr, b1, b2, eps,
                                   _stream(stream)), "igamg_adam_step")


def igamg_batch_create(dim, ps, ns):
    count = len(ps)
    pa = (ctypes.c_int * count)(*[int(v) for v in ps])
    na = (ctypes.c_int * count)(*[int(v) for v in ns])
    b = ctypes.c_void_p()
    _check(_load().igamg_batch_create(count, dim, pa, na, ctypes.byref(b)), "igamg_batch_create")
    return b


def igamg_batch_layout(batch, count):
    off = (ctypes.c_long * (count + 1))()
    _check(_load().igamg_batch_layout(batch, off), "igamg_batch_layout")
    return list(off)


def igamg_batch_workspace_bytes(batch, k, prec):
    return int(_load().igamg_batch_workspace_bytes(batch, k, prec))


def igamg_batch_rhs_sine(batch, coeffs, b, stream=None):
    """coeffs: array of shape (count, modes, ..., modes), one sine series per problem."""
    import numpy as np
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    _check(_load().igamg_batch_rhs_sine(batch, c.shape[1], _dbl(c), _ptr(b), _stream(stream)),
           "igamg_batch_rhs_sine")


def igamg_batch_solve(batch, count, b, x, tol, extrap, k, max_cycles, prec, ws, stream=None):
    """Returns (status, cycles[count], statuses[count], residuals[count])."""
    import numpy as np
    cyc = (ctypes.c_int * count)()
    st = (ctypes.c_int * count)()
    res = np.zeros(count)
    s = _load().igamg_batch_solve(batch, _ptr(b), _ptr(x), tol, extrap, k, max_cycles, prec, _ptr(ws),
                                  ws.numel(), _stream(stream), cyc, st, _dbl(res))
    if s not in (IGAMG_OK, IGAMG_ENOTCONV):
        _check(s, "igamg_batch_solve")
    return s, list(cyc), list(st), res


def igamg_batch_set_tail_ctas(batch, ctas):
    """Every problem's coarse tail on one CTA (1) or a cluster of 8 or 16 CTAs, at its deepest level."""
    _check(_load().igamg_batch_set_tail_ctas(batch, int(ctas)), "igamg_batch_set_tail_ctas")


def igamg_batch_set_device_loop(batch, enable):
    """Batched restart loops on the GPU in one graph (True) or as host-driven rounds (False)."""
    _check(_load().igamg_batch_set_device_loop(batch, 1 if enable else 0), "igamg_batch_set_device_loop")


def igamg_batch_destroy(batch):
    _load().igamg_batch_destroy(batch)


# ------------------------------------------------------------------ convenience
class Solver:
    """One problem: context + device workspace (a torch uint8 tensor)."""

    def __init__(self, dim, p, n, n_levels=0, k=10, prec="fp32_ir", device="cuda"):
        import torch
        self.dim, self.p = dim, p
        self.ctx = igamg_setup(dim, p, n, n_levels)
        igamg_assemble(self.ctx)
        self.levels = igamg_info(self.ctx)
        m = self.levels[-1]
        self.N = m[0] * m[1] * m[2]
        nbytes = max(igamg_workspace_bytes(self.ctx, k, v) for v in PREC.values())
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.k_max = k
        self.smoother = None

    def autotune(self, reps=3):
        """Pick the FP32 V-cycle launch schedule by timing (igamg_autotune)."""
        return igamg_autotune(self.ctx, self.ws, reps)

    def set_smoother(self, w, stall_ratio=0.95):
        """Use network weights w (device FP32 tensor, kept referenced here) as the
        learned post-smoother of prec='fp32_ir_learned' solves."""
        self.smoother = w
        igamg_set_smoother(self.ctx, w, stall_ratio)

    def rhs_sine(self, coeffs, b=None):
        import torch
        if b is None:
            b = torch.empty(self.N, dtype=torch.float64, device=self.ws.device)
        igamg_rhs_sine(self.ctx, coeffs, b)
        return b

    def solve(self, b, x=None, tol=1e-10, method="rre", k=5, max_cycles=200, prec="fp64",
              x0_given=False, absolute=False, graph=True, host_loop=False):
        import torch
        if x is None:
            x = torch.zeros(self.N, dtype=torch.float64, device=self.ws.device)
        flags = (IGAMG_FLAG_X0_GIVEN if x0_given else 0) | (IGAMG_FLAG_ABS_TOL if absolute else 0) | \
                (0 if graph else IGAMG_FLAG_NO_GRAPH) | (IGAMG_FLAG_HOST_LOOP if host_loop else 0)
        st, hist, cyc, vc = igamg_solve(self.ctx, b, x, tol, EXTRAP[method], k, max_cycles, PREC[prec],
                                        flags, self.ws)
        out = dict(x=x, status=st, history=hist, cycles=cyc, vcycles=vc, converged=st == IGAMG_OK)
        if prec == "fp32_ir_learned":
            out["fell_back"] = igamg_smoother_fell_back(self.ctx)
        return out

    def close(self):
        if self.ctx:
            igamg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GeneralSolver(Solver):
    """The full elliptic problem of Sec. 4.3 on a (mapped) unit square: the
    problem's functions are evaluated at the library's quadrature points
    (mapped by `geometry`, which returns (x, y, J)) and passed to the
    assembly; solves run in FP64."""

    def __init__(self, p, n, A, B, c, geometry=None, n_levels=0, k=10, device="cuda"):
        import numpy as np
        import torch
        self.dim, self.p = 2, p
        self.ctx = igamg_setup_general(p, n, n_levels)
        xi, eta = igamg_quadrature_points(self.ctx)
        if geometry is None:
            x, y, J = xi, eta, None
        else:
            x, y, J = geometry(xi, eta)
        self.points = (x, y)
        Av, Bv = A(x, y), B(x, y)
        coef = np.stack([Av[:, 0, 0], Av[:, 0, 1], Av[:, 1, 1], Bv[:, 0], Bv[:, 1], c(x, y)])
        jac = None if J is None else np.stack([J[:, 0, 0], J[:, 0, 1], J[:, 1, 0], J[:, 1, 1]])
        igamg_assemble_general(self.ctx, coef, jac)
        self.levels = igamg_info(self.ctx)
        m = self.levels[-1]
        self.N = m[0] * m[1] * m[2]
        self.ws = torch.empty(igamg_workspace_bytes(self.ctx, k, IGAMG_FP64), dtype=torch.uint8, device=device)
        self.k_max = k
        self.smoother = None

    def rhs(self, f):
        """Load vector of f (a function of the physical point)."""
        import torch
        b = torch.empty(self.N, dtype=torch.float64, device=self.ws.device)
        igamg_rhs_points(self.ctx, f(*self.points), b)
        return b


class Batch:
    """Many independent 2D/3D problems (degree p[i], n[i] elements per direction)
    solved together; vectors are packed back to back (see .offsets)."""

    def __init__(self, dim, ps, ns, k=5, device="cuda"):
        import torch
        self.count = len(ps)
        self.dim = dim
        self.handle = igamg_batch_create(dim, ps, ns)
        self.offsets = igamg_batch_layout(self.handle, self.count)
        self.N = self.offsets[-1]
        nbytes = max(igamg_batch_workspace_bytes(self.handle, k, PREC["fp32_ir"]),
                     igamg_batch_workspace_bytes(self.handle, k, PREC["fp64"]))
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.k_max = k

    def rhs_sine(self, coeffs):
        import torch
        b = torch.empty(self.N, dtype=torch.float64, device=self.ws.device)
        igamg_batch_rhs_sine(self.handle, coeffs, b)
        return b

    def autotune(self, reps=3):
        """Pick the FP32 V-cycle launch schedules by timing (igamg_batch_autotune)."""
        igamg_batch_autotune(self.handle, self.ws, reps)

    def solve(self, b, x=None, tol=1e-10, method="rre", k=5, max_cycles=200, prec="fp32_ir"):
        import torch
        if x is None:
            x = torch.empty(self.N, dtype=torch.float64, device=self.ws.device)
        st, cyc, sts, res = igamg_batch_solve(self.handle, self.count, b, x, tol, EXTRAP[method], k, max_cycles,
                                              PREC[prec], self.ws)
        return dict(x=x, status=st, cycles=cyc, statuses=sts, residuals=res, converged=st == IGAMG_OK)

    def close(self):
        if self.handle:
            igamg_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
