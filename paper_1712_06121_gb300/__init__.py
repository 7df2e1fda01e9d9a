"""Python binding of libcube (include/cube.h): CUBE's compressed-store
particle-mesh step on one GB300.

Argument marshalling only: every entry point has the C name and forwards to
the shared library; all work runs in the library's CUDA kernels.  Arrays may
be numpy arrays (host), torch tensors (host or CUDA), or raw integer
addresses.  Importing fails loudly if libcube.so has not been built.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcube.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libcube.so is not built ({LIB_PATH}); run "
                      "`python -m paper_1712_06121_gb300.build` (needs nvcc)")

_lib = ctypes.CDLL(LIB_PATH)

CUBE_OK, CUBE_E_ARG, CUBE_E_NOMEM, CUBE_E_CUDA, CUBE_E_STATE, CUBE_E_MIGRATION, \
    CUBE_E_OVERFLOW, CUBE_E_TIMEOUT = range(8)
STATUS_NAMES = ["CUBE_OK", "CUBE_E_ARG", "CUBE_E_NOMEM", "CUBE_E_CUDA", "CUBE_E_STATE",
                "CUBE_E_MIGRATION", "CUBE_E_OVERFLOW", "CUBE_E_TIMEOUT"]
CUBE_GRAD_FD4 = 0


class CubeError(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")


class cube_params(ctypes.Structure):
    _fields_ = [("n_fine", ctypes.c_int32), ("ratio", ctypes.c_int32), ("n_particles", ctypes.c_int64),
                ("x_bytes", ctypes.c_int32), ("v_bytes", ctypes.c_int32), ("id_bytes", ctypes.c_int32),
                ("gradient", ctypes.c_int32), ("deconv_power", ctypes.c_int32), ("brick", ctypes.c_int32),
                ("box", ctypes.c_double), ("omega_m", ctypes.c_double), ("omega_l", ctypes.c_double)]


class cube_state(ctypes.Structure):
    _fields_ = [("n_coarse", ctypes.c_int32), ("brick", ctypes.c_int32), ("x_bytes", ctypes.c_int32),
                ("v_bytes", ctypes.c_int32), ("id_bytes", ctypes.c_int32), ("n_particles", ctypes.c_int64),
                ("counts", ctypes.c_void_p), ("offsets", ctypes.c_void_p), ("vc", ctypes.c_void_p),
                ("chi", ctypes.c_void_p), ("nu", ctypes.c_void_p), ("id", ctypes.c_void_p),
                ("sigma", ctypes.c_double), ("a", ctypes.c_double), ("a_p", ctypes.c_double)]


class cube_stats(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("momentum", ctypes.c_double * 3), ("sigma", ctypes.c_double),
                ("a", ctypes.c_double), ("a_p", ctypes.c_double), ("steps", ctypes.c_int64),
                ("max_migration", ctypes.c_int32), ("error_flags", ctypes.c_uint32),
                ("last_step_ms", ctypes.c_double), ("kernel_launches", ctypes.c_int64),
                ("features", ctypes.c_uint32)]


class cube_step_limits(ctypes.Structure):
    _fields_ = [("drift_cells", ctypes.c_double), ("max_dlna", ctypes.c_double)]


class cube_memory_config(ctypes.Structure):
    _fields_ = [("x_bytes", ctypes.c_int32), ("v_bytes", ctypes.c_int32), ("id_bytes", ctypes.c_int32),
                ("ratio", ctypes.c_int32), ("coarse_per_image", ctypes.c_int32), ("buffer", ctypes.c_int32),
                ("tiles", ctypes.c_int32), ("eps_image", ctypes.c_double), ("eps_tile", ctypes.c_double),
                ("particles_per_image", ctypes.c_double)]


class cube_memory_layout(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("chi_nu", "chi_nu_tile", "ids", "rho_c", "v_c", "k_c", "k_f", "total")]


CUBE_PHASES = 12

CUBE_REQ_QUEUED, CUBE_REQ_RUNNING, CUBE_REQ_DONE, CUBE_REQ_FAILED = range(4)


class cube_request_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("steps_enqueued", ctypes.c_int32), ("n_steps", ctypes.c_int32),
                ("max_migration", ctypes.c_int32), ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("state_bytes", ctypes.c_int64), ("error", ctypes.c_int32)]


_P = ctypes.c_void_p
_sigs = {
    "cube_last_error": ([], ctypes.c_char_p),
    "cube_create": ([ctypes.POINTER(cube_params), _P, ctypes.POINTER(_P)], ctypes.c_int),
    "cube_destroy": ([_P], ctypes.c_int),
    "cube_encode": ([_P, _P, _P, _P, ctypes.c_double, ctypes.c_double], ctypes.c_int),
    "cube_pm_step": ([_P, ctypes.c_double, ctypes.c_double], ctypes.c_int),
    "cube_decode": ([_P, _P, _P, _P], ctypes.c_int),
    "cube_power_spectrum": ([_P, ctypes.c_int32, _P, _P, _P], ctypes.c_int),
    "cube_state_view": ([_P, ctypes.POINTER(cube_state)], ctypes.c_int),
    "cube_stats_get": ([_P, ctypes.POINTER(cube_stats)], ctypes.c_int),
    "cube_density": ([_P, _P], ctypes.c_int),
    "cube_potential": ([_P, _P], ctypes.c_int),
    "cube_keep_drifted": ([_P, ctypes.c_int32], ctypes.c_int),
    "cube_debug_drifted": ([_P, _P, _P, _P, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "cube_debug_force": ([_P, _P], ctypes.c_int),
    "cube_profile": ([_P, ctypes.c_int32], ctypes.c_int),
    "cube_profile_read": ([_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32),
                           ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "cube_phase_name": ([ctypes.c_int32], ctypes.c_char_p),
    "cube_counts_to_offsets_noalloc": ([_P, ctypes.c_int64, _P, _P], ctypes.c_int),
    "cube_max_speed": ([_P, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "cube_next_epoch": ([_P, ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "cube_max_force": ([_P, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "cube_next_epoch_limited": ([_P, ctypes.c_double, ctypes.POINTER(cube_step_limits), ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "cube_epoch_bound": ([ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                          ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.POINTER(cube_step_limits),
                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "cube_leapfrog_factors": ([ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "cube_memory_model": ([ctypes.POINTER(cube_memory_config), ctypes.POINTER(cube_memory_layout)], ctypes.c_int),
    "cube_counts_pack": ([_P, ctypes.c_int64, _P, _P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "cube_counts_unpack": ([_P, ctypes.c_int64, _P, ctypes.c_int64, _P], ctypes.c_int),
    "cube_checkpoint_size": ([ctypes.POINTER(cube_params), ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "cube_checkpoint_save": ([_P, _P], ctypes.c_int),
    "cube_checkpoint_load": ([_P, _P], ctypes.c_int),
    "cube_autotune_brick": ([ctypes.POINTER(cube_params), _P, _P, ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                             _P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "cube_server_sizes": ([ctypes.POINTER(cube_params), ctypes.POINTER(ctypes.c_int64),
                           ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "cube_server_create": ([ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_P)], ctypes.c_int),
    "cube_server_destroy": ([_P], ctypes.c_int),
    "cube_server_submit": ([_P, ctypes.POINTER(cube_params), _P, _P, _P, ctypes.c_double, _P, ctypes.c_int32,
                            ctypes.c_double, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "cube_server_pump": ([_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "cube_server_drain": ([_P], ctypes.c_int),
    "cube_server_info": ([_P, ctypes.c_int64, ctypes.POINTER(cube_request_info)], ctypes.c_int),
    "cube_server_result": ([_P, ctypes.c_int64, _P, _P, _P], ctypes.c_int),
    "cube_server_decode": ([_P, ctypes.c_int64, _P, _P, _P], ctypes.c_int),
    "cube_server_release": ([_P, ctypes.c_int64], ctypes.c_int),
    "cube_server_bytes": ([_P, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "cube_server_inject_alloc_failures": ([_P, ctypes.c_int32], ctypes.c_int),
    "cube_server_set_policy": ([_P, ctypes.c_int32], ctypes.c_int),
    "cube_batch_create": ([ctypes.POINTER(cube_params), ctypes.c_int32, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "cube_batch_destroy": ([_P], ctypes.c_int),
    "cube_batch_member": ([_P, ctypes.c_int32, ctypes.POINTER(_P)], ctypes.c_int),
    "cube_batch_step": ([_P, _P, _P], ctypes.c_int),
    "cube_batch_next_epochs": ([_P, _P, ctypes.c_double, _P], ctypes.c_int),
    "cube_batch_launches": ([_P, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "cube_batch_epochs_enqueue": ([_P], ctypes.c_int),
    "cube_batch_epochs_poll": ([_P, _P, ctypes.c_double, _P, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "cube_debug_velocity_tables": ([_P, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "cube_batch_solve": ([_P, _P], ctypes.c_int),
}
for _name, (_args, _res) in _sigs.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res


def _ptr(a):
    """Address of a numpy array / torch tensor / int (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if hasattr(a, "ctypes"):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"cannot take the address of {type(a)}")


def _check(status):
    if status != CUBE_OK:
        raise CubeError(status, cube_last_error())


def cube_last_error():
    return _lib.cube_last_error().decode()


def make_params(n_fine, n_particles, ratio=4, x_bytes=1, v_bytes=1, id_bytes=4, deconv_power=2,
                brick=0, box=100.0, omega_m=1.0, omega_l=0.0, gradient=CUBE_GRAD_FD4):
    return cube_params(n_fine, ratio, n_particles, x_bytes, v_bytes, id_bytes, gradient, deconv_power,
                       brick, box, omega_m, omega_l)


def cube_create(params, stream=None):
    """Returns the context handle.  `stream`: torch.cuda.Stream, raw handle or None."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    ctx = _P()
    _check(_lib.cube_create(ctypes.byref(params), stream, ctypes.byref(ctx)))
    return ctx


def cube_destroy(ctx):
    _check(_lib.cube_destroy(ctx))


def cube_encode(ctx, pos, vel, ids=None, a=0.02, sigma=0.0):
    _check(_lib.cube_encode(ctx, _ptr(pos), _ptr(vel), _ptr(ids), float(a), float(sigma)))


def cube_pm_step(ctx, a_from, a_to):
    _check(_lib.cube_pm_step(ctx, float(a_from), float(a_to)))


def cube_decode(ctx, pos, vel, ids=None):
    _check(_lib.cube_decode(ctx, _ptr(pos), _ptr(vel), _ptr(ids)))


def cube_power_spectrum(ctx, n_bins, k, pk, nmodes):
    _check(_lib.cube_power_spectrum(ctx, int(n_bins), _ptr(k), _ptr(pk), _ptr(nmodes)))


def cube_state_view(ctx):
    st = cube_state()
    _check(_lib.cube_state_view(ctx, ctypes.byref(st)))
    return st


def cube_stats_get(ctx):
    st = cube_stats()
    _check(_lib.cube_stats_get(ctx, ctypes.byref(st)))
    return st


def cube_max_speed(ctx):
    v = ctypes.c_double()
    _check(_lib.cube_max_speed(ctx, ctypes.byref(v)))
    return v.value


def cube_next_epoch(ctx, a_max, cells=0.5):
    v = ctypes.c_double()
    _check(_lib.cube_next_epoch(ctx, float(a_max), float(cells), ctypes.byref(v)))
    return v.value


def cube_max_force(ctx):
    v = ctypes.c_double()
    _check(_lib.cube_max_force(ctx, ctypes.byref(v)))
    return v.value


def cube_next_epoch_limited(ctx, a_max, drift_cells=0.5, max_dlna=0.0):
    """(a_to, binding): the largest a_to <= a_max within the drift limit (the
    fastest particle, kicked by the largest force of cube_max_force) and
    ln(a_to / a) <= max_dlna; binding 0 a_max, 1 drift, 2 expansion."""
    lim = cube_step_limits(float(drift_cells), float(max_dlna))
    out = ctypes.c_double()
    why = ctypes.c_int32()
    _check(_lib.cube_next_epoch_limited(ctx, float(a_max), ctypes.byref(lim), ctypes.byref(out), ctypes.byref(why)))
    return out.value, why.value


def cube_epoch_bound(omega_m, omega_l, ratio, a, a_p, a_max, p_max, f_max, drift_cells=0.5, max_dlna=0.0):
    """(a_to, binding) of cube_next_epoch_limited for given maxima, host only."""
    lim = cube_step_limits(float(drift_cells), float(max_dlna))
    out = ctypes.c_double()
    why = ctypes.c_int32()
    _check(_lib.cube_epoch_bound(float(omega_m), float(omega_l), int(ratio), float(a), float(a_p), float(a_max),
                                 float(p_max), float(f_max), ctypes.byref(lim), ctypes.byref(out), ctypes.byref(why)))
    return out.value, why.value


def cube_leapfrog_factors(omega_m, omega_l, a0, a1):
    """(kick, drift, growth_ratio) as the step evaluates them, host only."""
    k, d, g = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(_lib.cube_leapfrog_factors(float(omega_m), float(omega_l), float(a0), float(a1), ctypes.byref(k),
                                      ctypes.byref(d), ctypes.byref(g)))
    return k.value, d.value, g.value


def cube_density(ctx, rho):
    _check(_lib.cube_density(ctx, _ptr(rho)))


def cube_potential(ctx, phi):
    _check(_lib.cube_potential(ctx, _ptr(phi)))


def cube_keep_drifted(ctx, enable=True):
    _check(_lib.cube_keep_drifted(ctx, 1 if enable else 0))


def cube_debug_drifted(ctx, cell_old, u_new, p):
    s = ctypes.c_double()
    _check(_lib.cube_debug_drifted(ctx, _ptr(cell_old), _ptr(u_new), _ptr(p), ctypes.byref(s)))
    return s.value


def cube_debug_force(ctx, force):
    _check(_lib.cube_debug_force(ctx, _ptr(force)))


def cube_debug_velocity_tables(ctx):
    """(entries the kernels' compact 2-byte tables rebuild wrongly, entries they read whole)."""
    out = (ctypes.c_int64 * 2)()
    _check(_lib.cube_debug_velocity_tables(ctx, out))
    return int(out[0]), int(out[1])


def cube_profile(ctx, max_steps):
    _check(_lib.cube_profile(ctx, int(max_steps)))


def cube_profile_read(ctx):
    """Returns ({phase name: ms summed over traced steps}, {name: kernels per step}, steps)."""
    ms = (ctypes.c_double * CUBE_PHASES)()
    kn = (ctypes.c_int32 * CUBE_PHASES)()
    ns = ctypes.c_int32()
    _check(_lib.cube_profile_read(ctx, ms, kn, ctypes.byref(ns)))
    names = [cube_phase_name(i) for i in range(CUBE_PHASES)]
    return dict(zip(names, list(ms))), dict(zip(names, list(kn))), ns.value


def cube_counts_to_offsets_noalloc(counts, n_cells, offsets, stream=None):
    """Offsets of the cell-ordered store from per-cell counts, allocating nothing."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    _check(_lib.cube_counts_to_offsets_noalloc(_ptr(counts), int(n_cells), _ptr(offsets), stream))


def cube_phase_name(phase):
    return _lib.cube_phase_name(int(phase)).decode()


__all__ = [n for n in _sigs] + ["make_params", "cube_params", "cube_state", "cube_stats", "CubeError",
                                "LIB_PATH", "CUBE_GRAD_FD4", "CUBE_PHASES"]


def cube_memory_model(x_bytes=1, v_bytes=1, id_bytes=0, ratio=4, coarse_per_image=384, buffer=6, tiles=3,
                      eps_image=0.05, eps_tile=2.0, particles_per_image=1536.0 ** 3):
    """Bytes per image of each array of the paper's memory model, as a dict
    (host only; defaults are the configuration of its memory table)."""
    cfg = cube_memory_config(int(x_bytes), int(v_bytes), int(id_bytes), int(ratio), int(coarse_per_image),
                             int(buffer), int(tiles), float(eps_image), float(eps_tile), float(particles_per_image))
    out = cube_memory_layout()
    _check(_lib.cube_memory_model(ctypes.byref(cfg), ctypes.byref(out)))
    return {n: getattr(out, n) for n, _ in cube_memory_layout._fields_}


def cube_counts_pack(counts):
    """(bytes uint8[n], overflow uint32[k]) of host uint32 counts (Section 2.1's 1-byte field)."""
    import numpy as np
    c = np.ascontiguousarray(counts, dtype=np.uint32)
    b = np.empty(c.size, np.uint8)
    k = ctypes.c_int64()
    st = _lib.cube_counts_pack(c.ctypes.data, c.size, b.ctypes.data, None, 0, ctypes.byref(k))
    ov = np.empty(k.value, np.uint32)
    if st != CUBE_OK or k.value:
        _check(_lib.cube_counts_pack(c.ctypes.data, c.size, b.ctypes.data, ov.ctypes.data if k.value else None,
                                     k.value, ctypes.byref(k)))
    return b, ov


def cube_counts_unpack(bytes_, overflow):
    import numpy as np
    b = np.ascontiguousarray(bytes_, dtype=np.uint8)
    ov = np.ascontiguousarray(overflow, dtype=np.uint32)
    out = np.empty(b.size, np.uint32)
    _check(_lib.cube_counts_unpack(b.ctypes.data, b.size, ov.ctypes.data if ov.size else None, ov.size,
                                   out.ctypes.data))
    return out


def cube_checkpoint_size(params):
    v = ctypes.c_int64()
    _check(_lib.cube_checkpoint_size(ctypes.byref(params), ctypes.byref(v)))
    return v.value


def cube_checkpoint_save(ctx, buf):
    _check(_lib.cube_checkpoint_save(ctx, _ptr(buf)))


def cube_checkpoint_load(ctx, buf):
    _check(_lib.cube_checkpoint_load(ctx, _ptr(buf)))


def cube_autotune_brick(params, pos, vel, a, sigma, n_steps=5, stream=None):
    """(fastest brick side, [ms per step for bricks 1, 2, 4; -1 where invalid])."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    best = ctypes.c_int32()
    ms = (ctypes.c_double * 3)()
    _check(_lib.cube_autotune_brick(ctypes.byref(params), _ptr(pos), _ptr(vel), float(a), float(sigma),
                                    int(n_steps), stream, ctypes.byref(best), ms))
    return best.value, list(ms)


# ---------------------------------------------------------------- serving
def cube_server_sizes(params):
    """(state bytes, work bytes) of one request with these parameters."""
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.cube_server_sizes(ctypes.byref(params), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def cube_server_create(budget_bytes, n_streams=4, max_running=64):
    out = _P()
    _check(_lib.cube_server_create(int(budget_bytes), int(n_streams), int(max_running), ctypes.byref(out)))
    return out.value


def cube_server_destroy(srv):
    _check(_lib.cube_server_destroy(srv))


def cube_server_submit(srv, params, pos, vel, ids, sigma, epochs, n_bins, max_drift_cells=0.0):
    """Queues one simulation; epochs: n_steps + 1 increasing scale factors
    (copied); max_drift_cells > 0 makes them waypoints of velocity-limited
    steps.  pos, vel and ids must stay alive until the request is done.
    Returns the ticket."""
    import numpy as np
    ep = np.ascontiguousarray(epochs, dtype=np.float64)
    t = ctypes.c_int64()
    _check(_lib.cube_server_submit(srv, ctypes.byref(params), _ptr(pos), _ptr(vel), _ptr(ids), float(sigma),
                                   ep.ctypes.data, len(ep) - 1, float(max_drift_cells), int(n_bins),
                                   ctypes.byref(t)))
    return t.value


def cube_server_pump(srv):
    """Non-blocking progress; returns (running, queued)."""
    nr, nq = ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.cube_server_pump(srv, ctypes.byref(nr), ctypes.byref(nq)))
    return nr.value, nq.value


def cube_server_drain(srv):
    _check(_lib.cube_server_drain(srv))


def cube_server_info(srv, ticket):
    info = cube_request_info()
    _check(_lib.cube_server_info(srv, int(ticket), ctypes.byref(info)))
    return info


def cube_server_result(srv, ticket, k, pk, nmodes):
    _check(_lib.cube_server_result(srv, int(ticket), _ptr(k), _ptr(pk), _ptr(nmodes)))


def cube_server_decode(srv, ticket, pos, vel, ids):
    _check(_lib.cube_server_decode(srv, int(ticket), _ptr(pos), _ptr(vel), _ptr(ids)))


def cube_server_release(srv, ticket):
    _check(_lib.cube_server_release(srv, int(ticket)))


def cube_server_bytes(srv):
    v = ctypes.c_int64()
    _check(_lib.cube_server_bytes(srv, ctypes.byref(v)))
    return v.value


CUBE_ADMIT_FIFO, CUBE_ADMIT_SHORTEST = 0, 1


def cube_server_set_policy(srv, policy):
    _check(_lib.cube_server_set_policy(srv, int(policy)))


def cube_server_inject_alloc_failures(srv, n):
    _check(_lib.cube_server_inject_alloc_failures(srv, int(n)))


# ---------------------------------------------------------------- batches
def cube_batch_create(params_list, stream=None):
    """A batch of same-geometry simulations (list of cube_params); returns its handle."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    arr = (cube_params * len(params_list))(*params_list)
    b = _P()
    _check(_lib.cube_batch_create(arr, len(params_list), stream, ctypes.byref(b)))
    return b


def cube_batch_destroy(batch):
    _check(_lib.cube_batch_destroy(batch))


def cube_batch_member(batch, i):
    c = _P()
    _check(_lib.cube_batch_member(batch, int(i), ctypes.byref(c)))
    return c


def cube_batch_step(batch, a_from, a_to):
    import numpy as np
    af = np.ascontiguousarray(a_from, dtype=np.float64)
    at = np.ascontiguousarray(a_to, dtype=np.float64)
    _check(_lib.cube_batch_step(batch, af.ctypes.data, at.ctypes.data))


def cube_batch_solve(batch, stepping):
    """Enqueue the mesh half of the next batch step for the flagged members."""
    import numpy as np
    fl = np.ascontiguousarray(stepping, dtype=np.int32)
    _check(_lib.cube_batch_solve(batch, fl.ctypes.data))


def cube_batch_next_epochs(batch, a_max, cells=0.5):
    import numpy as np
    am = np.ascontiguousarray(a_max, dtype=np.float64)
    out = np.empty_like(am)
    _check(_lib.cube_batch_next_epochs(batch, am.ctypes.data, float(cells), out.ctypes.data))
    return out


def cube_batch_launches(batch):
    v = ctypes.c_int64()
    _check(_lib.cube_batch_launches(batch, ctypes.byref(v)))
    return v.value


def cube_batch_epochs_enqueue(batch):
    _check(_lib.cube_batch_epochs_enqueue(batch))


def cube_batch_epochs_poll(batch, a_max, cells=0.5):
    """None while the read-back is in flight, else the members' next epochs."""
    import numpy as np
    am = np.ascontiguousarray(a_max, dtype=np.float64)
    out = np.empty_like(am)
    ready = ctypes.c_int32()
    _check(_lib.cube_batch_epochs_poll(batch, am.ctypes.data, float(cells), out.ctypes.data, ctypes.byref(ready)))
    return out if ready.value else None
