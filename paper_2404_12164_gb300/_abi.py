"""ctypes mirror of include/fte.h and loader of libfte_gb300.so.

Loading fails loudly (ImportError) when the library is missing: there is no
fallback implementation.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfte_gb300.so")

FTE_NFIELD = 18
FTE_NCLASS = 32
FTE_REC = 24
FTE_HREC = 32
FTE_HHDR = 32
FTE_F32, FTE_BF16, FTE_F16 = range(3)
FTE_LAYOUT_CELL, FTE_LAYOUT_PAIR = 0, 1
FTE_MAX_OBS = 8
FTE_LEDGER = 8
FTE_MAX_SETS = 64
FTE_NGRAD = 5
FTE_LAYOUT_SHARED, FTE_LAYOUT_GLOBAL = 1, 2
FTE_OK, FTE_EINVAL, FTE_ENOMEM, FTE_ECUDA, FTE_ERANGE, FTE_ENOTSUP = range(6)
FTE_ALIVE, FTE_ABS_INNER, FTE_ABS_OUTER, FTE_ABS_THETA, FTE_DEAD_NAN, FTE_INJ_FAIL = range(6)
FTE_TALLY_S, FTE_TALLY_S2, FTE_TALLY_C, FTE_TALLY_INTENSITY = range(4)


class fte_grid(C.Structure):
    _fields_ = [("nr", C.c_int32), ("nth", C.c_int32), ("nph", C.c_int32), ("radial", C.c_int32),
                ("r_min", C.c_double), ("r_max", C.c_double),
                ("th_min", C.c_double), ("th_max", C.c_double),
                ("n_snap", C.c_int32), ("periodic", C.c_int32),
                ("t_snap0", C.c_double), ("dt_snap", C.c_double),
                ("dtype", C.c_int32), ("amr_levels", C.c_int32), ("amr_bsize", C.c_int32),
                ("n_leaves", C.c_int32), ("ring", C.c_int32), ("layout", C.c_int32)]


class fte_background(C.Structure):
    _fields_ = [("grid", fte_grid), ("fields", C.c_void_p), ("leaves", C.c_void_p),
                ("table", C.c_void_p)]


class fte_particles(C.Structure):
    _fields_ = [("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p), ("mu", C.c_void_p),
                ("p", C.c_void_p), ("w", C.c_void_p), ("id", C.c_void_p), ("status", C.c_void_p),
                ("capacity", C.c_uint64), ("count", C.c_uint64)]


class fte_inject_spec(C.Structure):
    _fields_ = [("region", C.c_int32), ("energy", C.c_int32), ("weight", C.c_int32),
                ("mu_mode", C.c_int32),
                ("r", C.c_double), ("th", C.c_double), ("ph", C.c_double),
                ("r1", C.c_double), ("r2", C.c_double), ("th1", C.c_double), ("th2", C.c_double),
                ("ph1", C.c_double), ("ph2", C.c_double),
                ("use_divv", C.c_int32), ("divv_snap", C.c_int32), ("max_tries", C.c_int32),
                ("pad0", C.c_int32), ("divv_max", C.c_double),
                ("e0", C.c_double), ("e1", C.c_double), ("e2", C.c_double), ("gamma", C.c_double),
                ("mu0", C.c_double), ("seed", C.c_uint32), ("set_id", C.c_uint32),
                ("id_base", C.c_uint32), ("pad1", C.c_uint32),
                ("spiral", C.c_double), ("spiral_rb", C.c_double)]


class fte_params(C.Structure):
    _fields_ = [("dmumu", C.c_int32), ("p_update", C.c_int32), ("kappa_drift", C.c_int32),
                ("dvdt_term", C.c_int32),
                ("lambda_par", C.c_double), ("p_ref", C.c_double), ("alpha", C.c_double),
                ("q", C.c_double), ("H", C.c_double), ("eps", C.c_double),
                ("mu_floor", C.c_double), ("lambda_perp", C.c_double),
                ("dt", C.c_double), ("t0", C.c_double),
                ("seed", C.c_uint32), ("set_id", C.c_uint32),
                ("sort_every", C.c_int32), ("tally_layout", C.c_int32)]


class fte_observer(C.Structure):
    _fields_ = [("kind", C.c_int32), ("ne", C.c_int32), ("nt", C.c_int32), ("pad", C.c_int32),
                ("r", C.c_double), ("dr", C.c_double), ("th", C.c_double), ("dth", C.c_double),
                ("ph", C.c_double), ("dph", C.c_double), ("e_lo", C.c_double), ("e_hi", C.c_double),
                ("t_lo", C.c_double), ("t_hi", C.c_double)]


class fte_tally_buf(C.Structure):
    _fields_ = [("n_obs", C.c_int32), ("n_sets", C.c_int32), ("obs", fte_observer * FTE_MAX_OBS),
                ("S", C.c_void_p), ("S2", C.c_void_p), ("C", C.c_void_p),
                ("ledger_w", C.c_void_p), ("ledger_n", C.c_void_p), ("S_class", C.c_void_p)]


class fte_smooth_obs(C.Structure):
    _fields_ = [("r_o", C.c_double), ("sigma_r", C.c_double), ("e_c", C.c_double), ("sigma_lnE", C.c_double),
                ("t_c", C.c_double), ("sigma_t", C.c_double), ("lr_window", C.c_double)]


class fte_set(C.Structure):
    _fields_ = [("lambda_par", C.c_double), ("q", C.c_double), ("H", C.c_double), ("eps", C.c_double),
                ("seed", C.c_uint32), ("set_id", C.c_uint32), ("count", C.c_uint64)]


class fte_launch_config(C.Structure):
    _fields_ = [("threads", C.c_int32), ("steps_per_launch", C.c_int32), ("tally_layout", C.c_int32),
                ("pad", C.c_int32)]


# every symbol include/fte.h declares, with its ctypes signature
_P = C.POINTER
SIGNATURES = {
    "fte_background_bytes": (C.c_size_t, [_P(fte_grid)]),
    "fte_load_background": (C.c_int, [_P(fte_grid), C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "fte_quantize_background": (C.c_int, [_P(fte_grid), C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "fte_amr_table_bytes": (C.c_size_t, [_P(fte_grid)]),
    "fte_amr_prepare": (C.c_int, [_P(fte_background), C.c_void_p]),
    "fte_tally_bins": (C.c_size_t, [_P(fte_tally_buf)]),
    "fte_tally_reset": (C.c_int, [_P(fte_tally_buf), C.c_void_p]),
    "fte_workspace_bytes": (C.c_size_t, [C.c_int, _P(fte_grid), _P(fte_tally_buf), C.c_uint64, C.c_int64]),
    "fte_inject": (C.c_int, [_P(fte_particles), _P(fte_background), _P(fte_inject_spec), C.c_uint64,
                             _P(fte_tally_buf), _P(C.c_uint64), C.c_void_p]),
    "fte_advance": (C.c_int, [_P(fte_particles), _P(fte_background), _P(fte_params),
                              _P(fte_tally_buf), C.c_int64, C.c_int64, C.c_void_p, C.c_size_t,
                              C.c_void_p]),
    "fte_advance_noalloc": (C.c_int, [_P(fte_particles), _P(fte_background), _P(fte_params),
                                      _P(fte_tally_buf), C.c_int64, C.c_int64, C.c_void_p]),
    "fte_tally": (C.c_int, [_P(fte_tally_buf), C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                            C.c_size_t, C.c_void_p]),
    "fte_tally_convolve": (C.c_int, [_P(fte_tally_buf), C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_size_t, C.c_void_p]),
    "fte_tally_set": (C.c_int, [_P(fte_tally_buf), C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                C.c_size_t, C.c_void_p]),
    "fte_workspace_bytes_batched": (C.c_size_t, [C.c_int, _P(fte_grid), _P(fte_tally_buf), C.c_uint64,
                                                 C.c_int64]),
    "fte_inject_batched": (C.c_int, [_P(fte_particles), _P(fte_background), _P(fte_inject_spec),
                                     _P(C.c_uint64), C.c_int, _P(fte_tally_buf), C.c_void_p]),
    "fte_advance_batched": (C.c_int, [_P(fte_particles), _P(fte_background), _P(fte_params), _P(fte_set),
                                      C.c_int, _P(fte_tally_buf), C.c_int64, C.c_int64,
                                      _P(fte_launch_config), C.c_void_p, C.c_size_t, C.c_void_p]),
    "fte_autotune_batched": (C.c_int, [_P(fte_particles), _P(fte_background), _P(fte_params), _P(fte_set),
                                       C.c_int, _P(fte_tally_buf), C.c_int64, C.c_int64, C.c_void_p,
                                       C.c_size_t, _P(fte_launch_config), _P(fte_launch_config),
                                       _P(C.c_double), _P(C.c_int), C.c_void_p]),
    "fte_adjoint_workspace_bytes": (C.c_size_t, [C.c_int, _P(fte_grid), C.c_uint64, C.c_int64, C.c_int]),
    "fte_adjoint_forward": (C.c_int, [_P(fte_particles), _P(fte_background), _P(fte_params), _P(fte_smooth_obs),
                                      C.c_int64, C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_size_t, C.c_void_p]),
    "fte_adjoint_reverse": (C.c_int, [_P(fte_particles), _P(fte_background), _P(fte_params), _P(fte_smooth_obs),
                                      _P(fte_inject_spec), C.c_int64, C.c_int64, C.c_int, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_size_t, C.c_void_p]),
    "fte_snapshot_bytes": (C.c_size_t, [_P(fte_grid)]),
    "fte_stream_staging_bytes": (C.c_size_t, [_P(fte_grid)]),
    "fte_stream_scales": (C.c_int, [_P(fte_background), C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "fte_stream_load": (C.c_int, [_P(fte_background), C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_size_t,
                                  C.c_void_p]),
    "fte_stream_plan": (C.c_int, [_P(fte_grid), _P(fte_params), C.c_int64, C.c_int64, C.c_void_p, C.c_int64,
                                  _P(C.c_int64)]),
    "fte_advance_streamed": (C.c_int, [_P(fte_particles), _P(fte_background), C.c_void_p, _P(fte_params),
                                       _P(fte_tally_buf), C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_size_t,
                                       C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p]),
    "fte_graph_begin": (C.c_int, [C.c_void_p]),
    "fte_graph_end": (C.c_int, [C.c_void_p, _P(C.c_void_p)]),
    "fte_graph_launch": (C.c_int, [C.c_void_p, C.c_void_p]),
    "fte_graph_destroy": (C.c_int, [C.c_void_p]),
    "fte_ledger": (C.c_int, [_P(fte_tally_buf), _P(C.c_double), _P(C.c_uint64), C.c_void_p]),
    "fte_probe_sectors": (C.c_int, [C.c_void_p, C.c_size_t, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "fte_probe_gather_l1": (C.c_int, [C.c_void_p, C.c_size_t, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                      C.c_void_p]),
    "fte_probe_step_timing": (C.c_int, [C.c_int]),
    "fte_probe_step_intervals": (C.c_int, [C.c_void_p, C.c_int, _P(C.c_int)]),
    "fte_last_error": (C.c_char_p, []),
    "fte_status_string": (C.c_char_p, [C.c_int]),
    "fte_abi_version": (C.c_int, []),
}

_lib = None


def lib():
    """The loaded library (raises ImportError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2404_12164_gb300/build.py "
                              "(or __graft_entry__.build()) first")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class FteError(RuntimeError):
    def __init__(self, status, where):
        L = lib()
        msg = L.fte_last_error().decode(errors="replace")
        super().__init__(f"{where}: {L.fte_status_string(status).decode()} ({status}): {msg}")
        self.status = status


def check(status, where):
    if status != FTE_OK:
        raise FteError(status, where)
    return status
