"""ctypes binding of the C ABI in include/mlmc.h (argument marshalling only).

Every function keeps the C name. Array arguments may be numpy arrays (host) or
torch tensors (host or CUDA); they must be contiguous and of the dtype the C
signature names (float64, int32, ...). All computation happens in the CUDA
library; importing this module fails loudly if the library was not built.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmlmc_gb300.so")

MLMC_OK = 0
MLMC_ERR_INVALID_ARG = 1
MLMC_ERR_OOM = 2
MLMC_ERR_CUDA = 3
MLMC_ERR_NOT_CONVERGED = 4
MLMC_ERR_TIMEOUT = 5
MLMC_ERR_UNIMPLEMENTED = 6
MLMC_PREC_FP64 = 0
MLMC_PREC_MIXED = 1

STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "NOT_CONVERGED", 5: "TIMEOUT",
                6: "UNIMPLEMENTED"}


class mlmc_config(ctypes.Structure):
    _fields_ = [
        ("lx", ctypes.c_double), ("ly", ctypes.c_double),
        ("nx0", ctypes.c_int32), ("ny0", ctypes.c_int32), ("levels", ctypes.c_int32),
        ("E11", ctypes.c_double), ("E22", ctypes.c_double), ("G12", ctypes.c_double),
        ("nu12", ctypes.c_double), ("E33", ctypes.c_double), ("nu13", ctypes.c_double),
        ("nu23", ctypes.c_double),
        ("kl_terms", ctypes.c_int32), ("kl_std", ctypes.c_double), ("kl_corr", ctypes.c_double),
        ("kl_quad", ctypes.c_int32),
        ("shortening", ctypes.c_double), ("omega_x0", ctypes.c_double), ("omega_x1", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("precision", ctypes.c_int32), ("rtol", ctypes.c_double),
        ("max_iter", ctypes.c_int32), ("max_outer", ctypes.c_int32), ("max_batch", ctypes.c_int64),
        ("mlmc_alpha", ctypes.c_double), ("mlmc_gamma", ctypes.c_double), ("mlmc_m", ctypes.c_double),
    ]


class mlmc_item(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int32), ("mesh_level", ctypes.c_int32), ("sample_id", ctypes.c_uint64)]


class mlmc_level_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("mean", ctypes.c_double * 2), ("m2", ctypes.c_double * 2),
                ("var", ctypes.c_double * 2), ("sum_qf", ctypes.c_double * 2),
                ("sum_qc", ctypes.c_double * 2), ("cost", ctypes.c_double)]

    def as_dict(self):
        return dict(n=self.n, mean=list(self.mean), m2=list(self.m2), var=list(self.var),
                    sum_qf=list(self.sum_qf), sum_qc=list(self.sum_qc), cost=self.cost)


SR_MAX_LEVELS = 16
REQ_SOLVE, REQ_SELECTIVE = 0, 1


class mlmc_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("level", ctypes.c_int32), ("mesh_level", ctypes.c_int32),
                ("sample_id", ctypes.c_uint64), ("tag", ctypes.c_uint64)]


class mlmc_result(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("kind", ctypes.c_int32), ("level", ctypes.c_int32),
                ("mesh_level", ctypes.c_int32), ("sample_id", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("q", ctypes.c_double * 2), ("stop_level", ctypes.c_int32),
                ("lambda_", ctypes.c_double * SR_MAX_LEVELS), ("lambda_fine", ctypes.c_double),
                ("lambda_coarse", ctypes.c_double), ("q_fine", ctypes.c_int32), ("q_coarse", ctypes.c_int32),
                ("solves", ctypes.c_int32), ("latency_ms", ctypes.c_double),
                ("pcg_iterations", ctypes.c_int32 * SR_MAX_LEVELS), ("q_mesh0", ctypes.c_int32)]

    def as_dict(self):
        return dict(tag=self.tag, kind=self.kind, level=self.level, mesh_level=self.mesh_level,
                    sample_id=self.sample_id, status=self.status, q=list(self.q), stop_level=self.stop_level,
                    lambdas=list(self.lambda_[:self.stop_level + 1]), lambda_fine=self.lambda_fine,
                    lambda_coarse=self.lambda_coarse, q_fine=self.q_fine, q_coarse=self.q_coarse,
                    solves=self.solves, latency_ms=self.latency_ms,
                    pcg_iterations=list(self.pcg_iterations[:min(self.solves, SR_MAX_LEVELS)]),
                    q_mesh0=self.q_mesh0)


class mlmc_server_config(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_int32), ("max_batch", ctypes.c_int64), ("hbm_budget_bytes", ctypes.c_double),
                ("threshold", ctypes.c_double), ("sr_factor", ctypes.c_double), ("eps_rel", ctypes.c_double),
                ("carry_iterates", ctypes.c_int32)]


_lib = None


def lib():
    """The loaded CUDA library (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run paper_1907_10271_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        P, I32, I64, U64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        sig = {
            "mlmc_create": (I32, [ctypes.POINTER(mlmc_config), P, ctypes.POINTER(P)]),
            "mlmc_destroy": (None, [P]),
            "mlmc_last_error": (ctypes.c_char_p, [P]),
            "mlmc_sample_level": (I32, [P, I32, U64, I64, P, P, P]),
            "mlmc_solve_batch": (I32, [P, P, I64, P, P]),
            "mlmc_estimate": (I32, [P, D, D, I64, I32, I32, P, P, P]),
            "mlmc_level_stats_get": (I32, [P, I32, P]),
            "mlmc_reset_stats": (I32, [P]),
            "mlmc_kl_coefficients": (I32, [P, I32, U64, I64, P]),
            "mlmc_theta": (I32, [P, I32, I32, U64, I64, P]),
            "mlmc_apply": (I32, [P, I32, I64, P, P, P]),
            "mlmc_solve_theta": (I32, [P, I32, I64, P, P, P, P]),
            "mlmc_sample_levels": (I32, [P, I32, P, P, P, P, P, P]),
            "mlmc_set_nested_threshold": (I32, [P, I64]),
            "mlmc_autotune": (I32, [P, I32, P, P, I32, P]),
            "mlmc_get_tuning": (I32, [P, P]),
            "mlmc_set_tuning": (I32, [P, P]),
            "mlmc_profile_enable": (I32, [P, I32]),
            "mlmc_profile_get": (I32, [P, I32, P, P, P]),
            "mlmc_launch_count": (I32, [P, P]),
            "mlmc_merge_stats": (I32, [P, P, P]),
            "mlmc_profile_report": (I32, [P, P, I64]),
            "mlmc_solve_theta_static": (I32, [ctypes.POINTER(mlmc_config), P, I32, I64, P, P, P]),
            "mlmc_static_last_error": (ctypes.c_char_p, []),
            "mlmc_server_create": (I32, [ctypes.POINTER(mlmc_config), ctypes.POINTER(mlmc_server_config),
                                         ctypes.POINTER(P)]),
            "mlmc_server_submit": (I32, [P, P, I64]),
            "mlmc_server_poll": (I32, [P, P, I64, P]),
            "mlmc_server_drain": (I32, [P, D]),
            "mlmc_server_counters": (I32, [P, P, P, P]),
            "mlmc_server_destroy": (None, [P]),
            "mlmc_server_last_error": (ctypes.c_char_p, [P]),
            "mlmc_failure_estimate": (I32, [P, I64, D, I32, I32, P, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class MLMCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(a, dtype):
    """Device or host address of a contiguous array of the given numpy dtype."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):          # torch tensor
        import torch
        tmap = {np.float64: torch.float64, np.float32: torch.float32, np.int32: torch.int32,
                np.int64: torch.int64, np.uint64: torch.uint64}
        if a.dtype != tmap[dtype] or not a.is_contiguous():
            raise TypeError(f"expected contiguous {dtype.__name__} tensor")
        return ctypes.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError(f"expected C-contiguous numpy {dtype.__name__} array")
    return ctypes.c_void_p(a.ctypes.data)


def _check(ctx, status):
    if status != MLMC_OK:
        msg = lib().mlmc_last_error(ctx).decode(errors="replace")
        raise MLMCError(status, msg)
    return status


def config_from_workload(w, **overrides):
    """mlmc_config from a workload dict (see workloads.py); keyword overrides win."""
    w = dict(w)
    w.update(overrides)
    c = mlmc_config()
    for f in ("lx", "ly", "E11", "E22", "G12", "nu12", "E33", "nu13", "nu23", "kl_corr", "shortening",
              "omega_x0", "omega_x1", "rtol"):
        setattr(c, f, float(w[f]))
    c.nx0, c.ny0, c.levels = int(w["nx0"]), int(w["ny0"]), int(w["levels"])
    c.kl_terms, c.kl_quad = int(w["kl_terms"]), int(w["kl_quad"])
    c.kl_std = float(np.deg2rad(w["kl_std_deg"]))
    c.seed = int(w["seed"])
    c.precision = MLMC_PREC_MIXED if w["precision"] == "mixed" else MLMC_PREC_FP64
    c.max_iter = int(w.get("max_iter", 0))
    c.max_outer = int(w.get("max_outer", 0))
    c.max_batch = int(w.get("max_batch", 0))
    c.mlmc_alpha = float(w.get("mlmc_alpha", 1.0))
    c.mlmc_gamma = float(w.get("mlmc_gamma", 1.0))
    c.mlmc_m = float(w.get("mlmc_m", 4.0))
    return c


def current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return 0


def mlmc_create(cfg, stream=None):
    h = ctypes.c_void_p()
    st = current_stream() if stream is None else stream
    s = lib().mlmc_create(ctypes.byref(cfg), ctypes.c_void_p(st), ctypes.byref(h))
    if s != MLMC_OK:
        raise MLMCError(s, lib().mlmc_last_error(None).decode(errors="replace"))
    return h


def mlmc_destroy(ctx):
    lib().mlmc_destroy(ctx)


def mlmc_last_error(ctx):
    return lib().mlmc_last_error(ctx).decode(errors="replace")


def mlmc_sample_level(ctx, level, first_id, n, q_fine=None, q_coarse=None, status=None):
    return _check(ctx, lib().mlmc_sample_level(ctx, level, first_id, n, _ptr(q_fine, np.float64),
                                                _ptr(q_coarse, np.float64), _ptr(status, np.int32)))


def mlmc_solve_batch(ctx, items, q=None, status=None):
    """items: sequence of (level, mesh_level, sample_id)."""
    arr = (mlmc_item * len(items))(*[mlmc_item(int(a), int(b), int(c)) for a, b, c in items])
    return _check(ctx, lib().mlmc_solve_batch(ctx, ctypes.cast(arr, ctypes.c_void_p), len(items),
                                               _ptr(q, np.float64), _ptr(status, np.int32)))


def mlmc_estimate(ctx, e, theta, n_star, max_level, qoi=0):
    """Returns (status, estimate, [level stats dicts], L)."""
    est = ctypes.c_double()
    L = ctypes.c_int32()
    stats = (mlmc_level_stats * (max_level + 1))()
    s = lib().mlmc_estimate(ctx, e, theta, n_star, max_level, qoi, ctypes.byref(est),
                            ctypes.cast(stats, ctypes.c_void_p), ctypes.byref(L))
    if s not in (MLMC_OK, MLMC_ERR_NOT_CONVERGED):
        _check(ctx, s)
    return s, est.value, [stats[i].as_dict() for i in range(L.value + 1)], L.value


def mlmc_level_stats_get(ctx, level):
    out = mlmc_level_stats()
    _check(ctx, lib().mlmc_level_stats_get(ctx, level, ctypes.byref(out)))
    return out.as_dict()


def mlmc_reset_stats(ctx):
    return _check(ctx, lib().mlmc_reset_stats(ctx))


def mlmc_kl_coefficients(ctx, level, first_id, n, xi):
    return _check(ctx, lib().mlmc_kl_coefficients(ctx, level, first_id, n, _ptr(xi, np.float64)))


def mlmc_theta(ctx, level, mesh_level, first_id, n, theta):
    return _check(ctx, lib().mlmc_theta(ctx, level, mesh_level, first_id, n, _ptr(theta, np.float64)))


def mlmc_apply(ctx, mesh_level, n, theta, p, q):
    return _check(ctx, lib().mlmc_apply(ctx, mesh_level, n, _ptr(theta, np.float64), _ptr(p, np.float64),
                                         _ptr(q, np.float64)))


def mlmc_solve_theta(ctx, mesh_level, n, theta, q, status=None, iterations=None):
    return _check(ctx, lib().mlmc_solve_theta(ctx, mesh_level, n, _ptr(theta, np.float64), _ptr(q, np.float64),
                                               _ptr(status, np.int32), _ptr(iterations, np.int32)))


def mlmc_sample_levels(ctx, levels, first_ids, counts, q_fine=None, q_coarse=None, status=None):
    """levels, first_ids, counts: sequences (host); outputs concatenated in request order."""
    n = len(levels)
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    fi = np.ascontiguousarray(first_ids, dtype=np.uint64)
    ct = np.ascontiguousarray(counts, dtype=np.int64)
    return _check(ctx, lib().mlmc_sample_levels(ctx, n, _ptr(lv, np.int32), _ptr(fi, np.uint64), _ptr(ct, np.int64),
                                                 _ptr(q_fine, np.float64), _ptr(q_coarse, np.float64),
                                                 _ptr(status, np.int32)))


PROFILE_OPS = ["pcg_update_presmooth", "presmooth", "postsmooth", "postsmooth_top", "search_direction",
               "refinement_residual", "coarsest", "other"]


# bits of mlmc_tuning.wide_strips (node-pair strip kernels)
MLMC_WIDE_PRE_TOP, MLMC_WIDE_PRE, MLMC_WIDE_POST, MLMC_WIDE_POST_TOP, MLMC_WIDE_SEARCH = 1, 2, 4, 8, 16
MLMC_WIDE_ALL = 31


class mlmc_tuning(ctypes.Structure):
    _fields_ = [("max_rows", ctypes.c_int32), ("min_rows", ctypes.c_int32), ("target_waves", ctypes.c_double),
                ("nested_min_nodes", ctypes.c_int64), ("fused_bottom", ctypes.c_int32), ("step_ms", ctypes.c_double),
                ("pack_samples", ctypes.c_int32), ("device_loop", ctypes.c_int32), ("wide_strips", ctypes.c_int32),
                ("omega", ctypes.c_double), ("omega_retries", ctypes.c_int64)]

    def as_dict(self):
        return dict(max_rows=self.max_rows, min_rows=self.min_rows, target_waves=self.target_waves,
                    nested_min_nodes=self.nested_min_nodes, fused_bottom=self.fused_bottom, step_ms=self.step_ms,
                    pack_samples=self.pack_samples, device_loop=self.device_loop, wide_strips=self.wide_strips,
                    omega=self.omega, omega_retries=self.omega_retries)


def mlmc_autotune(ctx, levels, counts, reps=2):
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    ct = np.ascontiguousarray(counts, dtype=np.int64)
    out = mlmc_tuning()
    _check(ctx, lib().mlmc_autotune(ctx, len(lv), _ptr(lv, np.int32), _ptr(ct, np.int64), reps, ctypes.byref(out)))
    return out.as_dict()


def mlmc_get_tuning(ctx):
    out = mlmc_tuning()
    _check(ctx, lib().mlmc_get_tuning(ctx, ctypes.byref(out)))
    return out.as_dict()


def mlmc_set_tuning(ctx, max_rows, min_rows, target_waves, nested_min_nodes, fused_bottom=1, pack_samples=1,
                    device_loop=0, wide_strips=None, omega=None):
    """wide_strips, omega None keep the context's current values."""
    cur = mlmc_get_tuning(ctx)
    if wide_strips is None:
        wide_strips = cur["wide_strips"]
    if omega is None:
        omega = cur["omega"]
    t = mlmc_tuning(max_rows, min_rows, target_waves, nested_min_nodes, fused_bottom, 0.0, pack_samples, device_loop,
                    wide_strips, omega, 0)
    return _check(ctx, lib().mlmc_set_tuning(ctx, ctypes.byref(t)))


def mlmc_set_nested_threshold(ctx, min_nodes):
    return _check(ctx, lib().mlmc_set_nested_threshold(ctx, int(min_nodes)))


def mlmc_profile_enable(ctx, on=True):
    return _check(ctx, lib().mlmc_profile_enable(ctx, 1 if on else 0))


def mlmc_profile_get(ctx, op):
    """(total ms, launches, nodes) of operation index `op` (see PROFILE_OPS)."""
    ms = ctypes.c_double()
    la = ctypes.c_int64()
    nd = ctypes.c_uint64()
    _check(ctx, lib().mlmc_profile_get(ctx, op, ctypes.byref(ms), ctypes.byref(la), ctypes.byref(nd)))
    return ms.value, la.value, nd.value


def mlmc_launch_count(ctx):
    n = ctypes.c_int64()
    _check(ctx, lib().mlmc_launch_count(ctx, ctypes.byref(n)))
    return n.value


def mlmc_solve_theta_static(cfg, mesh_level, n, theta, q, status=None, stream=None):
    """Allocation-free solve (no context): see include/mlmc.h."""
    st = current_stream() if stream is None else stream
    s = lib().mlmc_solve_theta_static(ctypes.byref(cfg), ctypes.c_void_p(st), mesh_level, n,
                                      _ptr(theta, np.float64), _ptr(q, np.float64), _ptr(status, np.int32))
    if s != MLMC_OK:
        raise MLMCError(s, lib().mlmc_static_last_error().decode(errors="replace"))
    return s


def stats_from_dict(d):
    s = mlmc_level_stats()
    s.n = int(d["n"])
    for k in range(2):
        s.mean[k], s.m2[k], s.var[k] = d["mean"][k], d["m2"][k], d["var"][k]
        s.sum_qf[k], s.sum_qc[k] = d["sum_qf"][k], d["sum_qc"][k]
    s.cost = d.get("cost", 0.0)
    return s


def mlmc_merge_stats(a, b):
    """Merged moments (dict) of two disjoint sample sets given as stats dicts."""
    out = mlmc_level_stats()
    sa, sb = stats_from_dict(a), stats_from_dict(b)
    s = lib().mlmc_merge_stats(ctypes.byref(sa), ctypes.byref(sb), ctypes.byref(out))
    if s != MLMC_OK:
        raise MLMCError(s, "merge")
    return out.as_dict()


def mlmc_profile_report(ctx):
    """{launch name: (launches, total ms)} since the last mlmc_profile_enable."""
    buf = ctypes.create_string_buffer(1 << 16)
    _check(ctx, lib().mlmc_profile_report(ctx, ctypes.cast(buf, ctypes.c_void_p), len(buf)))
    out = {}
    for line in buf.value.decode().splitlines():
        name, n, ms = line.rsplit(" ", 2)
        out[name] = (int(n), float(ms))
    return out


# ---------------------------------------------------------------- serving

def mlmc_server_create(cfg, workers=2, max_batch=4096, hbm_budget_bytes=8e9, threshold=0.0, sr_factor=2.0,
                       eps_rel=1e-6, carry_iterates=True):
    L = lib()
    sc = mlmc_server_config(workers, max_batch, float(hbm_budget_bytes), float(threshold), float(sr_factor),
                            float(eps_rel), 1 if carry_iterates else 0)
    srv = ctypes.c_void_p()
    st = L.mlmc_server_create(ctypes.byref(cfg), ctypes.byref(sc), ctypes.byref(srv))
    if st != 0:
        raise MLMCError(st, L.mlmc_server_last_error(None).decode())
    return srv


def mlmc_server_submit(srv, requests):
    """requests: iterable of (kind, level, mesh_level, sample_id, tag)."""
    reqs = list(requests)
    arr = (mlmc_request * max(1, len(reqs)))(*[mlmc_request(*r) for r in reqs])
    st = lib().mlmc_server_submit(srv, ctypes.cast(arr, ctypes.c_void_p), len(reqs))
    if st != 0:
        raise MLMCError(st, lib().mlmc_server_last_error(srv).decode())


def mlmc_server_poll(srv, max_results=4096):
    buf = (mlmc_result * max_results)()
    n = ctypes.c_int64()
    st = lib().mlmc_server_poll(srv, ctypes.cast(buf, ctypes.c_void_p), max_results, ctypes.byref(n))
    if st != 0:
        raise MLMCError(st, lib().mlmc_server_last_error(srv).decode())
    return [buf[k].as_dict() for k in range(n.value)]


def mlmc_server_drain(srv, timeout_ms=600000.0):
    """True when every submitted request completed within the timeout."""
    return lib().mlmc_server_drain(srv, float(timeout_ms)) == 0


def mlmc_server_counters(srv):
    b, s, pk = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    lib().mlmc_server_counters(srv, ctypes.byref(b), ctypes.byref(s), ctypes.byref(pk))
    return {"batches": b.value, "solves": s.value, "peak_bytes": pk.value}


def mlmc_server_last_error(srv):
    return lib().mlmc_server_last_error(srv).decode()


def mlmc_server_destroy(srv):
    lib().mlmc_server_destroy(srv)


def mlmc_failure_estimate(results, threshold, k=1, two_level=False):
    """(estimate, mean[16], var[16]) from result dicts of mlmc_server_poll."""
    arr = (mlmc_result * max(1, len(results)))()
    for i, r in enumerate(results):
        a = arr[i]
        a.tag, a.kind, a.level, a.mesh_level, a.sample_id = r["tag"], r["kind"], r["level"], r["mesh_level"], r["sample_id"]
        a.status, a.stop_level = r["status"], r["stop_level"]
        for j, v in enumerate(r["lambdas"]):
            a.lambda_[j] = v
        a.lambda_fine, a.lambda_coarse, a.q_fine, a.q_coarse = r["lambda_fine"], r["lambda_coarse"], r["q_fine"], r["q_coarse"]
        a.q_mesh0 = int(r.get("q_mesh0", 1 if r["lambdas"] and r["lambdas"][0] > threshold else 0))
    est = ctypes.c_double()
    mean = (ctypes.c_double * SR_MAX_LEVELS)()
    var = (ctypes.c_double * SR_MAX_LEVELS)()
    st = lib().mlmc_failure_estimate(ctypes.cast(arr, ctypes.c_void_p), len(results), float(threshold), int(k),
                                     1 if two_level else 0, ctypes.byref(est), ctypes.cast(mean, ctypes.c_void_p),
                                     ctypes.cast(var, ctypes.c_void_p))
    if st != 0:
        raise MLMCError(st, "mlmc_failure_estimate")
    return est.value, list(mean), list(var)


# ---------------------------------------------------------------- 3D Hex8 block (mlmc3d.h)

class mlmc3d_config(ctypes.Structure):
    _fields_ = [
        ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
        ("nx0", ctypes.c_int32), ("ny0", ctypes.c_int32), ("nz0", ctypes.c_int32), ("levels", ctypes.c_int32),
        ("E11", ctypes.c_double), ("E22", ctypes.c_double), ("E33", ctypes.c_double),
        ("G12", ctypes.c_double), ("G13", ctypes.c_double), ("G23", ctypes.c_double),
        ("nu12", ctypes.c_double), ("nu13", ctypes.c_double), ("nu23", ctypes.c_double),
        ("kl_terms", ctypes.c_int32), ("kl_std", ctypes.c_double), ("kl_corr", ctypes.c_double),
        ("kl_quad", ctypes.c_int32),
        ("shortening", ctypes.c_double), ("omega_x0", ctypes.c_double), ("omega_x1", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("rtol", ctypes.c_double),
        ("max_iter", ctypes.c_int32), ("max_outer", ctypes.c_int32),
    ]


_SIG3 = None


def lib3():
    """The library with the 3D entry points' signatures set."""
    global _SIG3
    L = lib()
    if _SIG3 is None:
        P, I32, I64, U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        sig = {
            "mlmc3d_create": (I32, [ctypes.POINTER(mlmc3d_config), P, ctypes.POINTER(P)]),
            "mlmc3d_destroy": (None, [P]),
            "mlmc3d_last_error": (ctypes.c_char_p, [P]),
            "mlmc3d_sample_level": (I32, [P, I32, U64, I64, P, P, P]),
            "mlmc3d_solve_batch": (I32, [P, P, I64, P, P]),
            "mlmc3d_level_stats_get": (I32, [P, I32, P]),
            "mlmc3d_reset_stats": (I32, [P]),
            "mlmc3d_theta": (I32, [P, I32, I32, U64, I64, P]),
            "mlmc3d_apply": (I32, [P, I32, I64, P, P, P]),
            "mlmc3d_apply_bench": (I32, [P, I32, I64, I32, P, P, P]),
            "mlmc3d_last_iters": (I32, [P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _SIG3 = True
    return L


def config3_from_workload(w, **overrides):
    """mlmc3d_config from a 3D workload dict (see workloads.py); keyword overrides win."""
    w = dict(w)
    w.update(overrides)
    c = mlmc3d_config()
    for f in ("lx", "ly", "lz", "E11", "E22", "E33", "G12", "G13", "G23", "nu12", "nu13", "nu23", "kl_corr",
              "shortening", "omega_x0", "omega_x1", "rtol"):
        setattr(c, f, float(w[f]))
    c.nx0, c.ny0, c.nz0, c.levels = int(w["nx0"]), int(w["ny0"]), int(w["nz0"]), int(w["levels"])
    c.kl_terms, c.kl_quad = int(w["kl_terms"]), int(w["kl_quad"])
    c.kl_std = float(np.deg2rad(w["kl_std_deg"]))
    c.seed = int(w["seed"])
    c.max_iter = int(w.get("max_iter", 0))
    c.max_outer = int(w.get("max_outer", 0))
    return c


def _check3(ctx, status):
    if status != MLMC_OK:
        raise MLMCError(status, lib3().mlmc3d_last_error(ctx).decode(errors="replace"))
    return status


def mlmc3d_create(cfg, stream=None):
    h = ctypes.c_void_p()
    st = current_stream() if stream is None else stream
    s = lib3().mlmc3d_create(ctypes.byref(cfg), ctypes.c_void_p(st), ctypes.byref(h))
    if s != MLMC_OK:
        raise MLMCError(s, lib3().mlmc3d_last_error(None).decode(errors="replace"))
    return h


def mlmc3d_destroy(ctx):
    lib3().mlmc3d_destroy(ctx)


def mlmc3d_sample_level(ctx, level, first_id, n, q_fine=None, q_coarse=None, status=None):
    return _check3(ctx, lib3().mlmc3d_sample_level(ctx, level, first_id, n, _ptr(q_fine, np.float64),
                                                    _ptr(q_coarse, np.float64), _ptr(status, np.int32)))


def mlmc3d_solve_batch(ctx, items, q=None, status=None):
    arr = (mlmc_item * len(items))(*[mlmc_item(int(l), int(m), int(s)) for (l, m, s) in items])
    return _check3(ctx, lib3().mlmc3d_solve_batch(ctx, ctypes.cast(arr, ctypes.c_void_p), len(items),
                                                   _ptr(q, np.float64), _ptr(status, np.int32)))


def mlmc3d_level_stats(ctx, level):
    out = mlmc_level_stats()
    _check3(ctx, lib3().mlmc3d_level_stats_get(ctx, level, ctypes.byref(out)))
    return out.as_dict()


def mlmc3d_reset_stats(ctx):
    return _check3(ctx, lib3().mlmc3d_reset_stats(ctx))


def mlmc3d_theta(ctx, mesh_level, level, first_id, n, theta):
    return _check3(ctx, lib3().mlmc3d_theta(ctx, mesh_level, level, first_id, n, _ptr(theta, np.float64)))


def mlmc3d_apply(ctx, mesh_level, n, theta, x, y):
    return _check3(ctx, lib3().mlmc3d_apply(ctx, mesh_level, n, _ptr(theta, np.float64), _ptr(x, np.float32),
                                             _ptr(y, np.float32)))


def mlmc3d_apply_bench(ctx, mesh_level, n, reps):
    ms, by, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check3(ctx, lib3().mlmc3d_apply_bench(ctx, mesh_level, n, reps, ctypes.byref(ms), ctypes.byref(by),
                                            ctypes.byref(fl)))
    return ms.value, by.value, fl.value


def mlmc3d_last_iters(ctx):
    it = ctypes.c_int32()
    _check3(ctx, lib3().mlmc3d_last_iters(ctx, ctypes.byref(it)))
    return it.value


# ---------------------------------------------------------------- panel buckling (mlmc_panel.h)

MLMCP_MAX_PLIES = 32


class mlmcp_config(ctypes.Structure):
    _fields_ = [
        ("lx", ctypes.c_double), ("ly", ctypes.c_double),
        ("nx0", ctypes.c_int32), ("ny0", ctypes.c_int32), ("levels", ctypes.c_int32),
        ("E11", ctypes.c_double), ("E22", ctypes.c_double), ("G12", ctypes.c_double), ("nu12", ctypes.c_double),
        ("G13", ctypes.c_double), ("k_shear", ctypes.c_double),
        ("n_plies", ctypes.c_int32), ("plies_deg", ctypes.c_double * MLMCP_MAX_PLIES),
        ("t_ply", ctypes.c_double), ("ply_std_deg", ctypes.c_double),
        ("hard_support", ctypes.c_int32), ("p_star", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
        ("smoother", ctypes.c_int32),
    ]


_SIGP = None


def libp():
    """The library with the panel entry points' signatures set."""
    global _SIGP
    L = lib()
    if _SIGP is None:
        P, I32, I64, U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        sig = {
            "mlmcp_create": (I32, [ctypes.POINTER(mlmcp_config), P, ctypes.POINTER(P)]),
            "mlmcp_destroy": (None, [P]),
            "mlmcp_last_error": (ctypes.c_char_p, [P]),
            "mlmcp_sample_level": (I32, [P, I32, U64, I64, P, P, P]),
            "mlmcp_solve_batch": (I32, [P, P, I64, P, P]),
            "mlmcp_level_stats_get": (I32, [P, I32, P]),
            "mlmcp_reset_stats": (I32, [P]),
            "mlmcp_laminate": (I32, [P, I32, U64, I64, P, P]),
            "mlmcp_apply": (I32, [P, I32, I32, U64, I64, P, P, P]),
            "mlmcp_last_iters": (I32, [P, P]),
            "mlmcp_apply_bench": (I32, [P, I32, I64, I32, P, P]),
            "mlmcp_server_create": (I32, [ctypes.POINTER(mlmcp_config), ctypes.POINTER(mlmc_server_config),
                                          ctypes.c_double, ctypes.c_double, ctypes.POINTER(P)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _SIGP = True
    return L


def configp_from_workload(w, **overrides):
    """mlmcp_config from a panel workload dict (see workloads.py); keyword overrides win."""
    w = dict(w)
    w.update(overrides)
    c = mlmcp_config()
    for f in ("lx", "ly", "E11", "E22", "G12", "nu12", "G13", "k_shear", "t_ply", "ply_std_deg", "p_star"):
        setattr(c, f, float(w[f]))
    c.nx0, c.ny0, c.levels = int(w["nx0"]), int(w["ny0"]), int(w["levels"])
    plies = list(w["plies_deg"])
    if not 1 <= len(plies) <= MLMCP_MAX_PLIES:
        raise ValueError("1 to 32 plies")
    c.n_plies = len(plies)
    for k, a in enumerate(plies):
        c.plies_deg[k] = float(a)
    c.hard_support = 1 if w.get("bc", "hard") == "hard" else 0
    c.seed = int(w["seed"])
    c.tol = float(w.get("tol", 0.0))
    c.max_iter = int(w.get("max_iter", 0))
    c.smoother = {"nodal": 0, "patch": 1}[w.get("smoother", "nodal")]
    return c


def _checkp(ctx, status):
    if status != MLMC_OK:
        raise MLMCError(status, libp().mlmcp_last_error(ctx).decode(errors="replace"))
    return status


def mlmcp_create(cfg, stream=None):
    h = ctypes.c_void_p()
    st = current_stream() if stream is None else stream
    s = libp().mlmcp_create(ctypes.byref(cfg), ctypes.c_void_p(st), ctypes.byref(h))
    if s != MLMC_OK:
        raise MLMCError(s, libp().mlmcp_last_error(None).decode(errors="replace"))
    return h


def mlmcp_destroy(ctx):
    libp().mlmcp_destroy(ctx)


def mlmcp_sample_level(ctx, level, first_id, n, q_fine=None, q_coarse=None, status=None):
    return _checkp(ctx, libp().mlmcp_sample_level(ctx, level, first_id, n, _ptr(q_fine, np.float64),
                                                   _ptr(q_coarse, np.float64), _ptr(status, np.int32)))


def mlmcp_solve_batch(ctx, items, q=None, status=None):
    arr = (mlmc_item * len(items))(*[mlmc_item(int(l), int(m), int(s)) for (l, m, s) in items])
    return _checkp(ctx, libp().mlmcp_solve_batch(ctx, ctypes.cast(arr, ctypes.c_void_p), len(items),
                                                  _ptr(q, np.float64), _ptr(status, np.int32)))


def mlmcp_level_stats(ctx, level):
    out = mlmc_level_stats()
    _checkp(ctx, libp().mlmcp_level_stats_get(ctx, level, ctypes.byref(out)))
    return out.as_dict()


def mlmcp_reset_stats(ctx):
    return _checkp(ctx, libp().mlmcp_reset_stats(ctx))


def mlmcp_laminate(ctx, level, first_id, n, dstar, kgt=None):
    return _checkp(ctx, libp().mlmcp_laminate(ctx, level, first_id, n, _ptr(dstar, np.float64),
                                               _ptr(kgt, np.float64)))


def mlmcp_apply(ctx, mesh_level, level, first_id, n, x, y, g=None):
    return _checkp(ctx, libp().mlmcp_apply(ctx, mesh_level, level, first_id, n, _ptr(x, np.float32),
                                            _ptr(y, np.float32), _ptr(g, np.float32)))


def mlmcp_apply_bench(ctx, mesh_level, n, reps=20):
    """(ms per launch, algorithmic bytes per launch) of the FP32 K / G operator kernel."""
    ms, by = ctypes.c_double(), ctypes.c_double()
    _checkp(ctx, libp().mlmcp_apply_bench(ctx, mesh_level, n, reps, ctypes.byref(ms), ctypes.byref(by)))
    return ms.value, by.value


def mlmcp_last_iters(ctx):
    it = ctypes.c_int32()
    _checkp(ctx, libp().mlmcp_last_iters(ctx, ctypes.byref(it)))
    return it.value


def mlmcp_server_create(cfg, workers=2, max_batch=4096, hbm_budget_bytes=8e9, threshold=0.0, sr_factor=2.0,
                        eps_rel=1e-6, mlmc_m=4.0, mlmc_alpha=1.0):
    """A request loop over panel samples (mlmcp_config cfg); the other mlmc_server_*
    calls of this module work on it. SELECTIVE requests refine on the critical load P
    (kN) and fail below `threshold`."""
    L = libp()
    sc = mlmc_server_config(workers, max_batch, float(hbm_budget_bytes), float(threshold), float(sr_factor),
                            float(eps_rel), 0)
    srv = ctypes.c_void_p()
    st = L.mlmcp_server_create(ctypes.byref(cfg), ctypes.byref(sc), float(mlmc_m), float(mlmc_alpha),
                               ctypes.byref(srv))
    if st != 0:
        raise MLMCError(st, L.mlmc_server_last_error(None).decode())
    return srv


# ---------------------------------------------------------------- Cosserat strength (mlmc_cosserat.h)

class mlmcc_config(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_double), ("omega_side", ctypes.c_double),
        ("omega1", ctypes.c_double), ("omega2", ctypes.c_double), ("kl_std", ctypes.c_double),
        ("d_fibre", ctypes.c_double), ("vf", ctypes.c_double), ("Ef", ctypes.c_double), ("Em", ctypes.c_double),
        ("Gf", ctypes.c_double), ("Gm", ctypes.c_double), ("nu12", ctypes.c_double), ("nu23", ctypes.c_double),
        ("R_ratio", ctypes.c_double), ("tau_y", ctypes.c_double), ("shortening", ctypes.c_double),
        ("n0", ctypes.c_int32), ("levels", ctypes.c_int32), ("kl_terms0", ctypes.c_int32),
        ("kl_terms_step", ctypes.c_int32), ("seed", ctypes.c_uint64), ("rtol", ctypes.c_double),
        ("max_iter", ctypes.c_int32),
    ]


_SIGC = None


def libc():
    """The library with the Cosserat entry points' signatures set."""
    global _SIGC
    L = lib()
    if _SIGC is None:
        P, I32, I64, U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        sig = {
            "mlmcc_create": (I32, [ctypes.POINTER(mlmcc_config), P, ctypes.POINTER(P)]),
            "mlmcc_destroy": (None, [P]),
            "mlmcc_last_error": (ctypes.c_char_p, [P]),
            "mlmcc_sample_level": (I32, [P, I32, U64, I64, P, P, P]),
            "mlmcc_sample_levels": (I32, [P, I32, P, P, P, P, P, P]),
            "mlmcc_solve_batch": (I32, [P, P, I64, P, P]),
            "mlmcc_level_stats_get": (I32, [P, I32, P]),
            "mlmcc_estimate": (I32, [P, ctypes.c_double, ctypes.c_double, I64, I32, I32, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, P, P, P]),
            "mlmcc_reset_stats": (I32, [P]),
            "mlmcc_field": (I32, [P, I32, I32, U64, I64, P]),
            "mlmcc_apply": (I32, [P, I32, I32, U64, I64, P, P]),
            "mlmcc_displacement": (I32, [P, I32, I32, U64, I64, P, P]),
            "mlmcc_last_iters": (I32, [P, P, P]),
            "mlmcc_launch_count": (I32, [P, P]),
            "mlmcc_profile_enable": (I32, [P, I32]),
            "mlmcc_profile_get": (I32, [P, I32, P, P, P]),
            "mlmcc_profile_name": (ctypes.c_char_p, [I32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _SIGC = True
    return L


def configc_from_workload(w, **overrides):
    """mlmcc_config from a Cosserat workload dict (see workloads.py); keyword overrides win."""
    w = dict(w)
    w.update(overrides)
    c = mlmcc_config()
    for f in ("L", "omega_side", "omega1", "omega2", "kl_std", "vf", "Ef", "Em", "Gf", "Gm", "nu12", "nu23",
              "R_ratio", "tau_y", "shortening"):
        setattr(c, f, float(w[f]))
    c.d_fibre = float(w["d"])
    c.n0, c.levels = int(w["n0"]), int(w["levels"])
    c.kl_terms0, c.kl_terms_step = int(w["kl_terms0"]), int(w["kl_terms_step"])
    c.seed = int(w["seed"])
    c.rtol = float(w.get("rtol", 0.0))
    c.max_iter = int(w.get("max_iter", 0))
    return c


def _checkc(ctx, status):
    if status != MLMC_OK:
        raise MLMCError(status, libc().mlmcc_last_error(ctx).decode(errors="replace"))
    return status


def mlmcc_create(cfg, stream=None):
    h = ctypes.c_void_p()
    st = current_stream() if stream is None else stream
    s = libc().mlmcc_create(ctypes.byref(cfg), ctypes.c_void_p(st), ctypes.byref(h))
    if s != MLMC_OK:
        raise MLMCError(s, libc().mlmcc_last_error(None).decode(errors="replace"))
    return h


def mlmcc_destroy(ctx):
    libc().mlmcc_destroy(ctx)


def mlmcc_sample_level(ctx, level, first_id, n, q_fine=None, q_coarse=None, status=None):
    return _checkc(ctx, libc().mlmcc_sample_level(ctx, level, first_id, n, _ptr(q_fine, np.float64),
                                                   _ptr(q_coarse, np.float64), _ptr(status, np.int32)))


def mlmcc_sample_levels(ctx, levels, first_ids, counts, q_fine=None, q_coarse=None, status=None):
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    fi = np.ascontiguousarray(first_ids, dtype=np.uint64)
    ct = np.ascontiguousarray(counts, dtype=np.int64)
    return _checkc(ctx, libc().mlmcc_sample_levels(ctx, len(lv), _ptr(lv, np.int32), _ptr(fi, np.uint64),
                                                    _ptr(ct, np.int64), _ptr(q_fine, np.float64),
                                                    _ptr(q_coarse, np.float64), _ptr(status, np.int32)))


def mlmcc_solve_batch(ctx, items, q=None, status=None):
    arr = (mlmc_item * len(items))(*[mlmc_item(int(l), int(m), int(s)) for (l, m, s) in items])
    return _checkc(ctx, libc().mlmcc_solve_batch(ctx, ctypes.cast(arr, ctypes.c_void_p), len(items),
                                                  _ptr(q, np.float64), _ptr(status, np.int32)))


def mlmcc_level_stats(ctx, level):
    out = mlmc_level_stats()
    _checkc(ctx, libc().mlmcc_level_stats_get(ctx, level, ctypes.byref(out)))
    return out.as_dict()


def mlmcc_estimate(ctx, e, theta=0.5, n_star=64, max_level=4, qoi=0, m=4.0, alpha=0.786, gamma=1.3):
    """Algorithm 1 on the Cosserat engine: (estimate, [level stats dicts], L, converged)."""
    stats = (mlmc_level_stats * (max_level + 1))()
    est, L = ctypes.c_double(), ctypes.c_int32()
    s = libc().mlmcc_estimate(ctx, float(e), float(theta), int(n_star), int(max_level), int(qoi), float(m),
                              float(alpha), float(gamma), ctypes.byref(est), ctypes.cast(stats, ctypes.c_void_p),
                              ctypes.byref(L))
    if s not in (MLMC_OK, MLMC_ERR_NOT_CONVERGED):
        _checkc(ctx, s)
    return est.value, [stats[l].as_dict() for l in range(L.value + 1)], L.value, s == MLMC_OK


def mlmcc_reset_stats(ctx):
    return _checkc(ctx, libc().mlmcc_reset_stats(ctx))


def mlmcc_field(ctx, level, mesh_level, first_id, n, phi):
    return _checkc(ctx, libc().mlmcc_field(ctx, level, mesh_level, first_id, n, _ptr(phi, np.float64)))


def mlmcc_apply(ctx, level, mesh_level, first_id, n, x, y):
    return _checkc(ctx, libc().mlmcc_apply(ctx, level, mesh_level, first_id, n, _ptr(x, np.float64),
                                            _ptr(y, np.float64)))


def mlmcc_displacement(ctx, level, mesh_level, first_id, n, d, status=None):
    return _checkc(ctx, libc().mlmcc_displacement(ctx, level, mesh_level, first_id, n, _ptr(d, np.float64),
                                                   _ptr(status, np.int32)))


def mlmcc_last_iters(ctx):
    it, rf = ctypes.c_int32(), ctypes.c_int32()
    _checkc(ctx, libc().mlmcc_last_iters(ctx, ctypes.byref(it), ctypes.byref(rf)))
    return it.value, rf.value


def mlmcc_launch_count(ctx):
    n = ctypes.c_int64()
    _checkc(ctx, libc().mlmcc_launch_count(ctx, ctypes.byref(n)))
    return n.value


def mlmcc_profile_enable(ctx, on=True):
    return _checkc(ctx, libc().mlmcc_profile_enable(ctx, 1 if on else 0))


def mlmcc_profile(ctx):
    """{kernel kind: (ms, launches, items)} accumulated since profiling was enabled."""
    out, k = {}, 0
    while True:
        name = libc().mlmcc_profile_name(k)
        if name is None:
            return out
        ms, la, it = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
        _checkc(ctx, libc().mlmcc_profile_get(ctx, k, ctypes.byref(ms), ctypes.byref(la), ctypes.byref(it)))
        if la.value:
            out[name.decode()] = (ms.value, la.value, it.value)
        k += 1
