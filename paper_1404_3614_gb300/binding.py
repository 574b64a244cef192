"""ctypes binding of libhomb (include/homb.h): argument marshalling only.

Every entry point keeps the C name. The functions take host structures built from a
``microstructures.Problem`` and raw device pointers (``tensor.data_ptr()``); torch is
used by callers only to own device memory and streams. There is no CPU fallback: if
the shared library cannot be loaded, importing the binding raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libhomb.so")

HOM_OK = 0
HOM_WARN_NOT_CONVERGED = 1
HOM_ERR_INVALID_ARG = -1
HOM_ERR_BREAKDOWN = -2
HOM_ERR_CUDA = -3
HOM_ERR_WORKSPACE = -4
HOM_ERR_TIMEOUT = -5
HOM_ERR_NOT_SPD_RESULT = -6

HOM_BOX, HOM_BALL = 0, 1
HOM_FP64, HOM_MIXED, HOM_FP32, HOM_FF = 0, 1, 2, 3
HOM_PRIMAL, HOM_DUAL = 0, 1


class hom_inclusion(C.Structure):
    _fields_ = [("shape", C.c_int32), ("reserved", C.c_int32), ("center", C.c_double * 3),
                ("size", C.c_double * 3), ("A", C.c_double * 9)]


class hom_problem(C.Structure):
    _fields_ = [("d", C.c_int32), ("N", C.c_int32 * 3), ("Y", C.c_double * 3), ("A0", C.c_double * 9),
                ("n_incl", C.c_int32), ("reserved", C.c_int32), ("incl", C.POINTER(hom_inclusion)),
                ("bitmap", C.POINTER(C.c_double)), ("bitmap_n", C.c_int32 * 3), ("closed", C.c_int32),
                ("smooth", C.c_int32)]


class hom_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("max_iter", C.c_int32), ("tol", C.c_double),
                ("check_every", C.c_int32), ("sides", C.c_int32), ("graph", C.c_int32),
                ("autotune", C.c_int32), ("dual_start", C.c_int32), ("discretization", C.c_int32),
                ("warm_start", C.c_int32), ("reserved", C.c_int32), ("net", C.c_void_p)]


class hom_report(C.Structure):
    _fields_ = [("iters", (C.c_int32 * 3) * 2), ("resid", (C.c_double * 3) * 2), ("matvecs", C.c_int32),
                ("status", (C.c_int32 * 3) * 2), ("ms_total", C.c_double), ("launches", C.c_int64),
                ("h2d_bytes", C.c_int64), ("d2h_bytes", C.c_int64), ("gani", (C.c_double * 9) * 2),
                ("batch_config", C.c_int32 * 6), ("elem_lo", C.c_double * 9), ("elem_hi", C.c_double * 9)]


class hom_field_io(C.Structure):
    _fields_ = [("d_x0", C.c_void_p), ("d_fields", C.c_void_p)]


class hom_batch_io(C.Structure):
    _fields_ = [("d_x0", C.c_void_p), ("d_fields", C.c_void_p)]


class hom_net_config(C.Structure):
    _fields_ = [("N", C.c_int32), ("cin", C.c_int32), ("width", C.c_int32), ("modes", C.c_int32),
                ("layers", C.c_int32), ("proj", C.c_int32), ("cout", C.c_int32), ("d", C.c_int32)]


class HombError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"homb status {status}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libhomb.so not built at {LIB_PATH}; run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    vp, sz, i32, i64, dp = C.c_void_p, C.c_size_t, C.c_int32, C.c_int64, C.POINTER(C.c_double)
    P = C.POINTER
    sigs = {
        "hom_create": (i32, [P(vp), C.c_int]),
        "hom_destroy": (i32, [vp]),
        "hom_last_error": (C.c_char_p, [vp]),
        "hom_version": (C.c_char_p, []),
        "hom_problem_info": (i32, [vp, P(hom_problem), P(i32), P(i32), P(i64), P(i64)]),
        "hom_workspace_size": (i32, [vp, P(hom_problem), P(hom_opts), P(sz)]),
        "hom_bounds": (i32, [vp, P(hom_problem), P(hom_opts), vp, sz, vp, dp, dp, dp, dp, P(hom_report)]),
        "hom_bounds_io": (i32, [vp, P(hom_problem), P(hom_opts), vp, sz, vp, dp, dp, dp, dp, P(hom_report),
                                P(hom_field_io)]),
        "hom_step_workspace_size": (i32, [vp, P(hom_problem), i32, P(sz)]),
        "hom_batched_workspace_size": (i32, [vp, i32, P(hom_problem), P(hom_opts), P(sz)]),
        "hom_bounds_batched": (i32, [vp, i32, P(hom_problem), P(hom_opts), vp, sz, vp, dp, dp, P(i32), P(i32),
                                     P(hom_report), P(hom_batch_io)]),
        "hom_net_sizes": (i32, [vp, P(hom_net_config), i32, P(i64), P(sz)]),
        "hom_net_init": (i32, [vp, P(hom_net_config), C.c_uint64, vp, vp]),
        "hom_net_forward": (i32, [vp, P(hom_net_config), vp, i32, vp, vp, vp, sz, vp]),
        "hom_net_gradient": (i32, [vp, P(hom_net_config), vp, i32, vp, vp, vp, P(C.c_float), vp, sz, vp]),
        "hom_net_train_step": (i32, [vp, P(hom_net_config), vp, vp, vp, vp, i32, C.c_float, i32, vp, vp, vp, vp,
                                     sz, vp]),
        "hom_net_features": (i32, [vp, i32, P(hom_problem), vp, vp, sz, vp]),
        "hom_grid_to_half": (i32, [vp, i32, i32, i32, i32, vp, vp, i32, vp]),
        "hom_half_to_grid_workspace_size": (i32, [vp, i32, i32, i32, i32, P(sz)]),
        "hom_resample_fields": (i32, [vp, i32, P(i32), P(i32), i64, i32, vp, vp, vp]),
        "hom_half_to_grid": (i32, [vp, i32, i32, i32, i32, vp, vp, i32, vp, sz, vp]),
        "hom_gemm_bf16": (i32, [vp, i32, i32, i32, vp, i32, i32, vp, i32, i32, vp, i32, C.c_float, C.c_float, vp]),
        "hom_coefficient": (i32, [vp, P(hom_problem), i32, i32, vp, vp, sz, vp]),
        "hom_rhs": (i32, [vp, P(hom_problem), i32, i32, i32, vp, vp, sz, vp]),
        "hom_matvec": (i32, [vp, P(hom_problem), i32, i32, i32, i32, vp, vp, vp, vp, sz, vp]),
        "hom_energy": (i32, [vp, P(hom_problem), i32, i32, vp, vp, dp, vp, sz, vp]),
        "hom_fft": (i32, [vp, i32, i32, i32, i32, vp, vp, vp, sz, vp]),
        "hom_matvec_noalloc": (i32, [vp, P(hom_problem), i32, i32, i32, i32, vp, vp, vp, vp]),
        "hom_set_pass_chunks": (i32, [vp, i32, i32]),
        "hom_set_slab_pass": (i32, [vp, i32]),
        "hom_set_batch_threads": (i32, [vp, i32]),
        "hom_set_batch_cluster": (i32, [vp, i32, i32]),
        "hom_profile_kernel": (i32, [vp, C.c_char_p]),
        "hom_kernel_timing": (i32, [vp, P(i64), dp]),
        "hom_peak_probe": (i32, [vp, i32, vp, dp]),
        "hom_set_gemm_spin_limit": (i32, [vp, i64]),
        "hom_set_net_chunk": (i32, [vp, i32]),
        "hom_set_pipe_passes": (i32, [vp, i32]),
        "hom_set_batch_warp_passes": (i32, [vp, i32]),
        "hom_set_inner_drift": (i32, [vp, C.c_double]),
        "hom_set_inner_floor": (i32, [vp, C.c_double]),
        "hom_set_refine_arith": (i32, [vp, i32]),
        "hom_energy_bounds": (i32, [vp, P(hom_problem), P(hom_opts), vp, sz, vp, dp, dp, dp, P(hom_report)]),
        "hom_net_save": (i32, [vp, P(hom_net_config), vp, C.c_char_p, vp]),
        "hom_net_load": (i32, [vp, C.c_char_p, P(vp)]),
        "hom_net_free": (i32, [vp]),
        "hom_net_info": (i32, [vp, P(hom_net_config), P(i64)]),
        "hom_net_normalise_targets": (i32, [vp, i32, i32, i32, vp, vp]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def declared_symbols():
    """Names of the functions the C header declares (parsed from include/homb.h)."""
    import re
    hdr = os.path.join(os.path.dirname(HERE), "include", "homb.h")
    src = open(hdr).read()
    return sorted(set(re.findall(r"^(?:hom_status|const char\*)\s+(hom_\w+)\s*\(", src, re.M)))


# ------------------------------------------------------------------------------------
# marshalling helpers
# ------------------------------------------------------------------------------------
def _mat3(A, d):
    out = np.zeros((3, 3))
    out[:d, :d] = np.asarray(A, dtype=np.float64)
    return out.reshape(-1)


def problem_struct(problem):
    """hom_problem from a microstructures.Problem. Returns (struct, keepalive)."""
    d = int(problem.d)
    n = len(problem.inclusions)
    arr = (hom_inclusion * max(n, 1))()
    for i, inc in enumerate(problem.inclusions):
        s = arr[i]
        s.shape = HOM_BOX if inc.shape == "box" else HOM_BALL
        c = np.zeros(3)
        c[:d] = inc.center
        sz = np.zeros(3)
        sz[:len(inc.size)] = inc.size
        s.center[:] = list(c)
        s.size[:] = list(sz)
        s.A[:] = list(_mat3(inc.A, d))
    p = hom_problem()
    p.d = d
    N = np.ones(3, dtype=np.int64)
    N[:d] = problem.N
    Y = np.ones(3)
    Y[:d] = problem.Y
    p.N[:] = [int(v) for v in N]
    p.Y[:] = [float(v) for v in Y]
    p.A0[:] = list(_mat3(problem.A0, d))
    p.n_incl = n
    p.incl = C.cast(arr, C.POINTER(hom_inclusion))
    keep = [arr]
    bm = getattr(problem, "bitmap", None)
    if bm is not None:
        # the ABI stores the x index fastest: the transpose of numpy's [i_1][i_2][(i_3)]
        img = np.ascontiguousarray(np.asarray(bm, dtype=np.float64).T)
        p.bitmap = img.ctypes.data_as(C.POINTER(C.c_double))
        P = [1, 1, 1]
        P[:d] = list(bm.shape)
        p.bitmap_n[:] = P
        keep.append(img)
    else:
        p.bitmap_n[:] = [1, 1, 1]
    p.closed = 1 if getattr(problem, "closed", False) else 0
    p.smooth = 1 if getattr(problem, "smooth", False) else 0
    return p, keep


def check(ctx, status, allow_warn=True):
    if status == HOM_OK or (allow_warn and status == HOM_WARN_NOT_CONVERGED):
        return status
    msg = lib.hom_last_error(ctx).decode() if ctx else ""
    raise HombError(status, msg)


def hom_create(device=0):
    h = C.c_void_p()
    st = lib.hom_create(C.byref(h), int(device))
    if st != HOM_OK:
        raise HombError(st, "hom_create failed (no CUDA device?)")
    return h


def hom_destroy(ctx):
    return lib.hom_destroy(ctx)


def hom_version():
    return lib.hom_version().decode()


def hom_last_error(ctx):
    return lib.hom_last_error(ctx).decode()


def hom_problem_info(ctx, problem):
    p, keep = problem_struct(problem)
    ncomp = C.c_int32()
    M = (C.c_int32 * 3)()
    fe = C.c_int64()
    ge = C.c_int64()
    check(ctx, lib.hom_problem_info(ctx, C.byref(p), C.byref(ncomp), M, C.byref(fe), C.byref(ge)))
    return {"ncomp": ncomp.value, "M": list(M), "field_elems": fe.value, "grid_elems": ge.value}


def make_opts(precision=HOM_FP64, tol=1e-8, max_iter=10000, check_every=8, sides=3, graph=0, autotune=0,
              dual_start=0, discretization=0, net=None):
    """hom_opts; `net` (a handle from hom_net_load) selects the learned warm start."""
    o = hom_opts()
    o.precision, o.tol, o.max_iter, o.check_every, o.sides = precision, tol, max_iter, check_every, sides
    o.graph, o.autotune, o.dual_start, o.discretization = graph, autotune, dual_start, discretization
    o.warm_start, o.net = (1, net) if net else (0, None)
    return o


def problems_array(problems):
    """A contiguous hom_problem[n] array (and the objects it points into)."""
    arr = (hom_problem * len(problems))()
    keep = []
    for i, pr in enumerate(problems):
        p, k = problem_struct(pr)
        arr[i] = p
        keep.append(k)
    return arr, keep


def hom_batched_workspace_size(ctx, problems, opts):
    arr, keep = problems_array(problems)
    n = C.c_size_t()
    check(ctx, lib.hom_batched_workspace_size(ctx, len(problems), arr, C.byref(opts), C.byref(n)))
    return n.value


def hom_bounds_batched(ctx, problems, opts, d_ws, ws_bytes, stream=0, d_x0=None, d_fields=None):
    """Returns dict(upper [n,2,2], lower [n,2,2], status [n], iters [n,2,2], report, code)."""
    arr, keep = problems_array(problems)
    n = len(problems)
    up = (C.c_double * (4 * n))()
    lo = (C.c_double * (4 * n))()
    stt = (C.c_int32 * n)()
    its = (C.c_int32 * (4 * n))()
    rep = hom_report()
    io = None
    if d_x0 is not None or d_fields is not None:
        io = hom_batch_io(C.c_void_p(d_x0 or 0), C.c_void_p(d_fields or 0))
    code = lib.hom_bounds_batched(ctx, n, arr, C.byref(opts), C.c_void_p(d_ws), ws_bytes, C.c_void_p(stream),
                                  up, lo, stt, its, C.byref(rep), C.byref(io) if io is not None else None)
    check(ctx, code)
    return {"upper": np.array(up[:]).reshape(n, 2, 2), "lower": np.array(lo[:]).reshape(n, 2, 2),
            "status": np.array(stt[:]), "iters": np.array(its[:]).reshape(n, 2, 2), "code": code,
            "report": {"ms_total": rep.ms_total, "launches": rep.launches, "h2d_bytes": rep.h2d_bytes,
                       "d2h_bytes": rep.d2h_bytes,
                       "config": dict(zip(("threads", "cap", "radix_schedule", "cluster", "coop_min_M", "ctas"),
                                          list(rep.batch_config)))}}


def hom_bounds_io(ctx, problem, opts, d_ws, ws_bytes, stream=0, d_x0=None, d_fields=None):
    """hom_bounds with starting / converged fields (device pointers, see hom_field_io)."""
    return hom_bounds(ctx, problem, opts, d_ws, ws_bytes, stream, d_x0, d_fields)


def hom_workspace_size(ctx, problem, opts):
    p, keep = problem_struct(problem)
    n = C.c_size_t()
    check(ctx, lib.hom_workspace_size(ctx, C.byref(p), C.byref(opts), C.byref(n)))
    return n.value


def hom_step_workspace_size(ctx, problem, nrhs):
    p, keep = problem_struct(problem)
    n = C.c_size_t()
    check(ctx, lib.hom_step_workspace_size(ctx, C.byref(p), int(nrhs), C.byref(n)))
    return n.value


def hom_bounds(ctx, problem, opts, d_ws, ws_bytes, stream=0, d_x0=None, d_fields=None):
    """Returns dict(upper, lower, mean, D, report, status) with d x d numpy arrays. d_x0 /
    d_fields: optional device pointers to starting / converged fields (hom_bounds_io)."""
    p, keep = problem_struct(problem)
    d = int(problem.d)
    bufs = {k: (C.c_double * (d * d))() for k in ("upper", "lower", "mean", "D")}
    rep = hom_report()
    if d_x0 is None and d_fields is None:
        st = lib.hom_bounds(ctx, C.byref(p), C.byref(opts), C.c_void_p(d_ws), ws_bytes, C.c_void_p(stream),
                            bufs["upper"], bufs["lower"], bufs["mean"], bufs["D"], C.byref(rep))
    else:
        io = hom_field_io(C.c_void_p(d_x0 or 0), C.c_void_p(d_fields or 0))
        st = lib.hom_bounds_io(ctx, C.byref(p), C.byref(opts), C.c_void_p(d_ws), ws_bytes, C.c_void_p(stream),
                               bufs["upper"], bufs["lower"], bufs["mean"], bufs["D"], C.byref(rep), C.byref(io))
    check(ctx, st)
    out = {k: np.array(v[:]).reshape(d, d) for k, v in bufs.items()}
    out["status"] = st
    out["report"] = {
        "iters": [list(rep.iters[s]) for s in range(2)],
        "resid": [list(rep.resid[s]) for s in range(2)],
        "status": [list(rep.status[s]) for s in range(2)],
        "matvecs": rep.matvecs, "ms_total": rep.ms_total, "launches": rep.launches,
        "h2d_bytes": rep.h2d_bytes, "d2h_bytes": rep.d2h_bytes,
    }
    if opts.discretization == 1:
        out["gani_A"] = np.array(rep.gani[0][:d * d]).reshape(d, d)
        out["gani_B"] = np.array(rep.gani[1][:d * d]).reshape(d, d)
    if (opts.sides or 3) & 3 == 3:
        out["elem_lo"] = np.array(rep.elem_lo[:d * d]).reshape(d, d)
        out["elem_hi"] = np.array(rep.elem_hi[:d * d]).reshape(d, d)
    return out


def hom_coefficient(ctx, problem, side, precision, d_coef, d_ws, ws_bytes, stream=0):
    p, keep = problem_struct(problem)
    return check(ctx, lib.hom_coefficient(ctx, C.byref(p), side, precision, C.c_void_p(d_coef),
                                          C.c_void_p(d_ws), ws_bytes, C.c_void_p(stream)))


def hom_rhs(ctx, problem, side, precision, nrhs, d_b, d_ws, ws_bytes, stream=0):
    p, keep = problem_struct(problem)
    return check(ctx, lib.hom_rhs(ctx, C.byref(p), side, precision, nrhs, C.c_void_p(d_b),
                                  C.c_void_p(d_ws), ws_bytes, C.c_void_p(stream)))


def hom_matvec(ctx, problem, side, precision, project, nrhs, d_coef, d_in, d_out, d_ws, ws_bytes, stream=0):
    p, keep = problem_struct(problem)
    return check(ctx, lib.hom_matvec(ctx, C.byref(p), side, precision, project, nrhs, C.c_void_p(d_coef),
                                     C.c_void_p(d_in), C.c_void_p(d_out), C.c_void_p(d_ws), ws_bytes,
                                     C.c_void_p(stream)))


def hom_matvec_noalloc(ctx, problem, side, precision, project, nrhs, d_coef, d_in, d_out, stream=0):
    """hom_matvec with the library's own static device scratch (no workspace argument)."""
    p, keep = problem_struct(problem)
    return check(ctx, lib.hom_matvec_noalloc(ctx, C.byref(p), side, precision, project, nrhs,
                                             C.c_void_p(d_coef), C.c_void_p(d_in), C.c_void_p(d_out),
                                             C.c_void_p(stream)))


HOM_NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024


def hom_energy(ctx, problem, nrhs, add_constant, d_coef, d_x, d_ws, ws_bytes, stream=0):
    p, keep = problem_struct(problem)
    W = (C.c_double * (nrhs * nrhs))()
    check(ctx, lib.hom_energy(ctx, C.byref(p), nrhs, add_constant, C.c_void_p(d_coef), C.c_void_p(d_x), W,
                              C.c_void_p(d_ws), ws_bytes, C.c_void_p(stream)))
    return np.array(W[:]).reshape(nrhs, nrhs)


def hom_fft(ctx, M, precision, direction, howmany, d_in, d_out, d_ws, ws_bytes, stream=0):
    return check(ctx, lib.hom_fft(ctx, M, precision, direction, howmany, C.c_void_p(d_in), C.c_void_p(d_out),
                                  C.c_void_p(d_ws), ws_bytes, C.c_void_p(stream)))


def hom_set_batch_threads(ctx, threads):
    return check(ctx, lib.hom_set_batch_threads(ctx, int(threads)))


def hom_set_batch_warp_passes(ctx, enable):
    """Warp-owned pencil passes in the FP32 iterations of batches (1, the default) or not (0)."""
    return check(ctx, lib.hom_set_batch_warp_passes(ctx, int(enable)))


def hom_set_batch_cluster(ctx, cluster, coop_min_M=0):
    return check(ctx, lib.hom_set_batch_cluster(ctx, int(cluster), int(coop_min_M)))


def hom_set_pass_chunks(ctx, ypass_pencils=0, xpass_planes=0):
    """Pencils per CTA of the operator's y passes and planes per CTA of its row pass (0: auto)."""
    return check(ctx, lib.hom_set_pass_chunks(ctx, ypass_pencils, xpass_planes))


def hom_set_slab_pass(ctx, enable):
    return check(ctx, lib.hom_set_slab_pass(ctx, int(enable)))


def hom_profile_kernel(ctx, name):
    return check(ctx, lib.hom_profile_kernel(ctx, (name or "").encode()))


def hom_kernel_timing(ctx):
    n = C.c_int64()
    ms = C.c_double()
    check(ctx, lib.hom_kernel_timing(ctx, C.byref(n), C.byref(ms)))
    return n.value, ms.value


def hom_energy_bounds(ctx, problem, opts, d_ws, ws_bytes, E, stream=0):
    """(E.A_up E, E.inv(B_up) E) for the host vector E (length d)."""
    p, keep = problem_struct(problem)
    Ev = (C.c_double * 3)(*[float(e) for e in E])
    up, lo = C.c_double(), C.c_double()
    rep = hom_report()
    check(ctx, lib.hom_energy_bounds(ctx, C.byref(p), C.byref(opts), C.c_void_p(d_ws), ws_bytes, C.c_void_p(stream),
                                     Ev, C.byref(up), C.byref(lo), C.byref(rep)))
    return up.value, lo.value


def hom_net_save(ctx, cfg, d_params, path, stream=0):
    return check(ctx, lib.hom_net_save(ctx, C.byref(cfg), C.c_void_p(d_params), os.fsencode(path), C.c_void_p(stream)))


def hom_net_load(ctx, path):
    """A host-side network handle (free it with hom_net_free)."""
    h = C.c_void_p()
    check(ctx, lib.hom_net_load(ctx, os.fsencode(path), C.byref(h)))
    return h.value


def hom_net_free(net):
    return lib.hom_net_free(C.c_void_p(net))


def hom_net_info(net):
    cfg = hom_net_config()
    n = C.c_int64()
    if lib.hom_net_info(C.c_void_p(net), C.byref(cfg), C.byref(n)) != HOM_OK:
        raise HombError(HOM_ERR_INVALID_ARG, "invalid network handle")
    return cfg, n.value


def hom_net_normalise_targets(ctx, d, N, n, d_grid, stream=0):
    return check(ctx, lib.hom_net_normalise_targets(ctx, int(d), int(N), int(n), C.c_void_p(d_grid),
                                                    C.c_void_p(stream)))


def hom_set_gemm_spin_limit(ctx, polls):
    """Test aid: the GEMMs of this context poll their completion barrier at most `polls`
    times (0: default)."""
    return check(ctx, lib.hom_set_gemm_spin_limit(ctx, int(polls)))


def hom_set_pipe_passes(ctx, enable):
    """Persistent pipelined FP32 z passes at length 225: mask 1 last pass (default), 2 z inverse,
    4 wide chunks of the last pass."""
    return check(ctx, lib.hom_set_pipe_passes(ctx, int(enable)))


def hom_set_inner_drift(ctx, c):
    """Drift coefficient c of the FP32 inner target of HOM_MIXED (0: the default)."""
    return check(ctx, lib.hom_set_inner_drift(ctx, float(c)))


def hom_set_inner_floor(ctx, eta):
    """Relative floor eta of the FP32 inner target of HOM_MIXED (0: the default, 1e-5)."""
    return check(ctx, lib.hom_set_inner_floor(ctx, float(eta)))


def hom_set_refine_arith(ctx, mode):
    """Residual arithmetic of HOM_MIXED's refinement steps: 1 FP64, 2 float-float, 0 the default."""
    return check(ctx, lib.hom_set_refine_arith(ctx, int(mode)))


def hom_set_net_chunk(ctx, cells):
    """Cells per network forward in the learned start of a batch (0: as many as fit 512 MiB)."""
    return check(ctx, lib.hom_set_net_chunk(ctx, int(cells)))


def hom_peak_probe(ctx, precision, stream=0):
    """Measured FMA rate (TFLOP/s) of this GPU in HOM_FP32 or HOM_FP64."""
    t = C.c_double()
    check(ctx, lib.hom_peak_probe(ctx, precision, stream, C.byref(t)))
    return t.value


# ------------------------------------------------------------------------------------
# learned warm start
# ------------------------------------------------------------------------------------
def net_config(N, cin=1, width=32, modes=12, layers=4, proj=128, cout=8, d=2):
    return hom_net_config(N, cin, width, modes, layers, proj, cout, d)


def hom_net_sizes(ctx, cfg, batch):
    n = C.c_int64()
    b = C.c_size_t()
    check(ctx, lib.hom_net_sizes(ctx, C.byref(cfg), batch, C.byref(n), C.byref(b)))
    return n.value, b.value


def hom_net_init(ctx, cfg, seed, d_params, stream=0):
    return check(ctx, lib.hom_net_init(ctx, C.byref(cfg), seed, C.c_void_p(d_params), C.c_void_p(stream)))


def hom_net_forward(ctx, cfg, d_params, batch, d_in, d_out, d_ws, ws_bytes, stream=0):
    return check(ctx, lib.hom_net_forward(ctx, C.byref(cfg), C.c_void_p(d_params), batch, C.c_void_p(d_in),
                                          C.c_void_p(d_out), C.c_void_p(d_ws), ws_bytes, C.c_void_p(stream)))


def hom_net_gradient(ctx, cfg, d_params, batch, d_in, d_target, d_grad, d_ws, ws_bytes, stream=0):
    loss = C.c_float()
    check(ctx, lib.hom_net_gradient(ctx, C.byref(cfg), C.c_void_p(d_params), batch, C.c_void_p(d_in),
                                    C.c_void_p(d_target), C.c_void_p(d_grad), C.byref(loss), C.c_void_p(d_ws),
                                    ws_bytes, C.c_void_p(stream)))
    return loss.value


def hom_net_train_step(ctx, cfg, d_params, d_m, d_v, d_grad, step, lr, batch, d_in, d_target, d_loss, d_ws,
                       ws_bytes, stream=0):
    return check(ctx, lib.hom_net_train_step(ctx, C.byref(cfg), C.c_void_p(d_params), C.c_void_p(d_m),
                                             C.c_void_p(d_v), C.c_void_p(d_grad), step, lr, batch,
                                             C.c_void_p(d_in), C.c_void_p(d_target), C.c_void_p(d_loss),
                                             C.c_void_p(d_ws), ws_bytes, C.c_void_p(stream)))


def hom_net_features(ctx, problems, d_features, d_ws, ws_bytes, stream=0):
    arr, keep = problems_array(problems)
    return check(ctx, lib.hom_net_features(ctx, len(problems), arr, C.c_void_p(d_features), C.c_void_p(d_ws),
                                           ws_bytes, C.c_void_p(stream)))


def hom_grid_to_half(ctx, d, N, batch, ch, d_grid, d_half, precision, stream=0):
    return check(ctx, lib.hom_grid_to_half(ctx, d, N, batch, ch, C.c_void_p(d_grid), C.c_void_p(d_half), precision,
                                           C.c_void_p(stream)))


def hom_resample_fields(ctx, d, N_from, N_to, count, precision, d_in, d_out, stream=0):
    f = (C.c_int32 * 3)(*(list(N_from) + [1] * (3 - len(N_from))))
    t = (C.c_int32 * 3)(*(list(N_to) + [1] * (3 - len(N_to))))
    return check(ctx, lib.hom_resample_fields(ctx, d, f, t, count, precision, C.c_void_p(d_in), C.c_void_p(d_out),
                                              C.c_void_p(stream)))


def hom_half_to_grid_workspace_size(ctx, d, N, batch, ch):
    b = C.c_size_t()
    check(ctx, lib.hom_half_to_grid_workspace_size(ctx, d, N, batch, ch, C.byref(b)))
    return b.value


def hom_half_to_grid(ctx, d, N, batch, ch, d_half, d_grid, precision, d_ws=0, ws_bytes=0, stream=0):
    return check(ctx, lib.hom_half_to_grid(ctx, d, N, batch, ch, C.c_void_p(d_half), C.c_void_p(d_grid), precision,
                                           C.c_void_p(d_ws), ws_bytes, C.c_void_p(stream)))


def hom_gemm_bf16(ctx, M, N, K, d_A, lda, ta, d_B, ldb, tb, d_C, ldc, alpha=1.0, beta=0.0, stream=0):
    return check(ctx, lib.hom_gemm_bf16(ctx, M, N, K, C.c_void_p(d_A), lda, ta, C.c_void_p(d_B), ldb, tb,
                                        C.c_void_p(d_C), ldc, alpha, beta, C.c_void_p(stream)))
