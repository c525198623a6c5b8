"""ctypes binding of libac (include/ac.h): same names, argument marshalling only.

Every step of the simulation runs in the CUDA kernels of ``libac.so``; this
module converts Python values and numpy / torch buffers into the C ABI's plain
pointers and sizes and turns non-zero statuses into :class:`ACError`.  If the
shared library is missing the import fails loudly -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# AC_LIB_PATH selects another build of the library (the bounds-checked libac_check.so)
LIB_PATH = os.environ.get("AC_LIB_PATH") or os.path.join(_PKG, "libac.so")

AC_OK, AC_ERR_ARG, AC_ERR_OOM, AC_ERR_CUDA, AC_ERR_STALL, AC_ERR_STATE = range(6)
AC_INIT_RANDOM, AC_INIT_UP, AC_INIT_DOWN = 0, 1, 2
AC_KERNEL_ROUND, AC_KERNEL_BLOCKED, AC_KERNEL_EPOCH = 0, 1, 2
AC_OPT_WATCHDOG_NS, AC_OPT_MAX_ROUNDS, AC_OPT_DROP_PUBLISH, AC_OPT_EARLY_REJECT = 1, 2, 3, 4
TICKS_PER_UNIT = 1 << 32

_STATUS = {AC_ERR_ARG: "AC_ERR_ARG", AC_ERR_OOM: "AC_ERR_OOM", AC_ERR_CUDA: "AC_ERR_CUDA",
           AC_ERR_STALL: "AC_ERR_STALL", AC_ERR_STATE: "AC_ERR_STATE"}


class ACError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class ac_lattice(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int32), ("cols", ctypes.c_int32), ("init", ctypes.c_int32)]


class ac_stats_t(ctypes.Structure):
    _fields_ = [("events", ctypes.c_uint64), ("rounds", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("scanned", ctypes.c_uint64), ("enabled", ctypes.c_uint64), ("visits", ctypes.c_uint64),
                ("polls", ctypes.c_uint64), ("global_rounds", ctypes.c_uint64),
                ("device_ms", ctypes.c_double), ("enabled_frac_mean", ctypes.c_double),
                ("sum_s", ctypes.c_int64), ("sum_bonds", ctypes.c_int64), ("checksum", ctypes.c_uint64),
                ("total_counts", ctypes.c_uint64), ("t_done", ctypes.c_int64),
                ("kernel", ctypes.c_int32), ("Lb", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("rounds_per_launch", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("early_commits", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


EXPORTS = ["ac_create", "ac_set_stream", "ac_configure", "ac_run_until", "ac_run_until_ticks",
           "ac_read_state", "ac_read_state_device", "ac_load_state", "ac_stats", "ac_round_history",
           "ac_destroy", "ac_last_error", "ac_thresholds", "ac_reset", "ac_set_option", "ac_batch_create", "ac_batch_run_until",
           "ac_dev_exp_ticks", "ac_dev_philox", "ac_run_blocked_static", "ac_frames_configure",
           "ac_run_until_frames", "ac_frames_status", "ac_time_model", "ac_create_life", "ac_set_rates",
           "ac_create_q", "ac_class_counts", "ac_load_state_async", "ac_read_state_async", "ac_slab_configure",
           "ac_slab_step", "ac_slab_export", "ac_slab_import"]

AC_RATE_ONE = 1 << 20

AC_LIFE_CONWAY_BIRTH, AC_LIFE_CONWAY_SURVIVE = 1 << 3, (1 << 2) | (1 << 3)

AC_LAW_EXP, AC_LAW_UNIFORM, AC_LAW_ROOT8 = 0, 1, 2

AC_MAX_FRAMES = 64
# void (*ac_frame_fn)(void* user, int64_t K, const int8_t* frame, size_t n)
FRAME_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t)


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libac.so not found at {path}: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    P, I32, I64, U64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    sig = {
        "ac_create": ([ac_lattice, D, D, D, U64, ctypes.POINTER(P)], I32),
        "ac_set_stream": ([P, P], I32),
        "ac_configure": ([P, I32, I32, I32, I32], I32),
        "ac_run_until": ([P, D], I32),
        "ac_run_until_ticks": ([P, I64], I32),
        "ac_read_state": ([P, P, P, P], I32),
        "ac_read_state_device": ([P, P, P, P], I32),
        "ac_load_state": ([P, P, P, P, I64], I32),
        "ac_load_state_async": ([P, P, P, P, I64, P], I32),
        "ac_slab_configure": ([P, I32, I32], I32),
        "ac_slab_step": ([P, I64, ctypes.POINTER(I32)], I32),
        "ac_slab_export": ([P, I32, I32, P], I32),
        "ac_slab_import": ([P, I32, I32, P], I32),
        "ac_read_state_async": ([P, P, P, P, P], I32),
        "ac_stats": ([P, ctypes.POINTER(ac_stats_t)], I32),
        "ac_round_history": ([P, P, I32, ctypes.POINTER(I32)], I32),
        "ac_destroy": ([P], None),
        "ac_reset": ([P, U64, I32], I32),
        "ac_set_option": ([P, I32, I64], I32),
        "ac_last_error": ([], ctypes.c_char_p),
        "ac_thresholds": ([D, D, D, P], I32),
        "ac_batch_create": ([I32, P, P, P, P, P, P], I32),
        "ac_batch_run_until": ([I32, P, P], I32),
        "ac_dev_exp_ticks": ([P, P, I64], I32),
        "ac_dev_philox": ([U64, P, P, ctypes.c_uint32, P, I64], I32),
        "ac_run_blocked_static": ([I32, I32, D, D, D, U64, P, P, I64, P], I32),
        "ac_frames_configure": ([P, I64, I64, I32], I32),
        "ac_run_until_frames": ([P, I64, FRAME_FN, P, I32], I32),
        "ac_frames_status": ([P, ctypes.POINTER(I64), ctypes.POINTER(I32), ctypes.POINTER(I64)], I32),
        "ac_set_rates": ([P, P], I32),
        "ac_class_counts": ([P, P], I32),
        "ac_create_q": ([ac_lattice, D, D, D, I32, U64, ctypes.POINTER(P)], I32),
        "ac_create_life": ([ac_lattice, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, U64,
                            ctypes.POINTER(P)], I32),
        "ac_time_model": ([I32, I64, I32, I32, U64, I64, I32, P, ctypes.POINTER(I32), P, P,
                           ctypes.POINTER(ctypes.c_double)], I32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = load_library()


def _check(status: int) -> None:
    if status != AC_OK:
        raise ACError(status, _lib.ac_last_error().decode(errors="replace"))


def _np_ptr(a: np.ndarray, dtype) -> ctypes.c_void_p:
    if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError(f"expected a C-contiguous {np.dtype(dtype).name} array")
    return ctypes.c_void_p(a.ctypes.data)


# ----------------------------------------------------------- same-name wrappers
def ac_create(rows: int, cols: int, init: int, beta: float, J: float, h: float, seed: int) -> int:
    out = ctypes.c_void_p()
    _check(_lib.ac_create(ac_lattice(rows, cols, init), beta, J, h, seed & (2**64 - 1), ctypes.byref(out)))
    return out.value


def ac_create_life(rows: int, cols: int, init: int, density: int, birth: int, survive: int, seed: int) -> int:
    out = ctypes.c_void_p()
    _check(_lib.ac_create_life(ac_lattice(rows, cols, init), int(density) & 0xFFFFFFFF, int(birth), int(survive),
                               seed & (2**64 - 1), ctypes.byref(out)))
    return out.value


def ac_create_q(rows: int, cols: int, init: int, beta: float, J: float, h: float, q: int, seed: int) -> int:
    out = ctypes.c_void_p()
    _check(_lib.ac_create_q(ac_lattice(rows, cols, init), beta, J, h, int(q), seed & (2**64 - 1), ctypes.byref(out)))
    return out.value


def ac_class_counts(sim: int) -> np.ndarray:
    """Cells per BKL class, index j + 5 (s > 0) (j up neighbours)."""
    out = np.zeros(10, dtype=np.uint64)
    _check(_lib.ac_class_counts(sim, _np_ptr(out, np.uint64)))
    return out


def ac_set_rates(sim: int, m) -> None:
    """Per-cell rates 2^20 / m[c] (None: rate 1 everywhere); only at time 0."""
    if m is None:
        _check(_lib.ac_set_rates(sim, None))
    else:
        _check(_lib.ac_set_rates(sim, _np_ptr(np.ascontiguousarray(m, dtype=np.uint32), np.uint32)))


def ac_set_stream(sim: int, stream: int) -> None:
    _check(_lib.ac_set_stream(sim, stream))


def ac_configure(sim: int, kernel: int, Lb: int, rounds: int, polls: int) -> None:
    _check(_lib.ac_configure(sim, kernel, Lb, rounds, polls))


def ac_run_until(sim: int, T: float) -> None:
    _check(_lib.ac_run_until(sim, float(T)))


def ac_run_until_ticks(sim: int, t_end: int) -> None:
    _check(_lib.ac_run_until_ticks(sim, int(t_end)))


def ac_read_state(sim: int, s: np.ndarray | None, t: np.ndarray | None, n: np.ndarray | None) -> None:
    _check(_lib.ac_read_state(sim, None if s is None else _np_ptr(s, np.int8),
                              None if t is None else _np_ptr(t, np.int64),
                              None if n is None else _np_ptr(n, np.uint32)))


def ac_read_state_device(sim: int, s_ptr: int | None, t_ptr: int | None, n_ptr: int | None) -> None:
    _check(_lib.ac_read_state_device(sim, s_ptr, t_ptr, n_ptr))


def ac_load_state(sim: int, s: np.ndarray, t: np.ndarray, n: np.ndarray, t_done: int) -> None:
    _check(_lib.ac_load_state(sim, _np_ptr(s, np.int8), _np_ptr(t, np.int64), _np_ptr(n, np.uint32),
                              int(t_done)))


def ac_load_state_async(sim: int, s: np.ndarray, t: np.ndarray, n: np.ndarray, t_done: int, stream) -> None:
    """Enqueue a state load on `stream` (a cudaStream_t as an int, or None); the host arrays (pinned
    for a truly asynchronous copy) must stay alive until the stream has passed this point."""
    _check(_lib.ac_load_state_async(sim, _np_ptr(s, np.int8), _np_ptr(t, np.int64), _np_ptr(n, np.uint32),
                                    int(t_done), stream))


def ac_read_state_async(sim: int, s: np.ndarray | None, t: np.ndarray | None, n: np.ndarray | None,
                        stream) -> None:
    """Enqueue a state read into host arrays on `stream`; they hold the state once the stream is done."""
    _check(_lib.ac_read_state_async(sim, None if s is None else _np_ptr(s, np.int8),
                                    None if t is None else _np_ptr(t, np.int64),
                                    None if n is None else _np_ptr(n, np.uint32), stream))


def ac_slab_configure(sim: int, row0: int, nrows: int) -> None:
    _check(_lib.ac_slab_configure(sim, int(row0), int(nrows)))


def ac_slab_step(sim: int, t_end: int) -> bool:
    """One temporal-blocked step of the handle's row slab; True if the slab is still live."""
    live = ctypes.c_int32(0)
    _check(_lib.ac_slab_step(sim, int(t_end), ctypes.byref(live)))
    return bool(live.value)


def ac_slab_export(sim: int, row: int, count: int, dst_ptr: int) -> None:
    _check(_lib.ac_slab_export(sim, int(row), int(count), dst_ptr))


def ac_slab_import(sim: int, row: int, count: int, src_ptr: int) -> None:
    _check(_lib.ac_slab_import(sim, int(row), int(count), src_ptr))


def ac_stats(sim: int) -> dict:
    st = ac_stats_t()
    _check(_lib.ac_stats(sim, ctypes.byref(st)))
    return st.as_dict()


def ac_round_history(sim: int) -> np.ndarray:
    n = ctypes.c_int32()
    _check(_lib.ac_round_history(sim, None, 0, ctypes.byref(n)))
    buf = np.zeros(max(n.value, 1), dtype=np.uint64)
    _check(_lib.ac_round_history(sim, _np_ptr(buf, np.uint64), n.value, ctypes.byref(n)))
    return buf[:n.value].copy()


def ac_destroy(sim: int) -> None:
    _lib.ac_destroy(sim)


def ac_reset(sim: int, seed: int, init: int) -> None:
    _check(_lib.ac_reset(sim, seed & (2**64 - 1), init))


def ac_set_option(sim: int, option: int, value: int) -> None:
    _check(_lib.ac_set_option(sim, option, int(value)))


def ac_thresholds(beta: float, J: float = 1.0, h: float = 0.0) -> np.ndarray:
    out = np.zeros(10, dtype=np.uint32)
    _check(_lib.ac_thresholds(beta, J, h, _np_ptr(out, np.uint32)))
    return out


def ac_batch_create(lattices, betas, Js, hs, seeds) -> list[int]:
    n = len(lattices)
    lats = (ac_lattice * n)(*[ac_lattice(r, c, i) for (r, c, i) in lattices])
    b = np.ascontiguousarray(betas, dtype=np.float64)
    j = np.ascontiguousarray(Js, dtype=np.float64)
    h = np.ascontiguousarray(hs, dtype=np.float64)
    s = np.ascontiguousarray([int(x) & (2**64 - 1) for x in seeds], dtype=np.uint64)
    out = (ctypes.c_void_p * n)()
    _check(_lib.ac_batch_create(n, ctypes.cast(lats, ctypes.c_void_p), _np_ptr(b, np.float64),
                                _np_ptr(j, np.float64), _np_ptr(h, np.float64), _np_ptr(s, np.uint64),
                                ctypes.cast(out, ctypes.c_void_p)))
    return [out[i] for i in range(n)]


def ac_batch_run_until(sims, t_end) -> None:
    n = len(sims)
    arr = (ctypes.c_void_p * n)(*sims)
    te = np.ascontiguousarray([int(x) for x in t_end], dtype=np.int64)
    _check(_lib.ac_batch_run_until(n, ctypes.cast(arr, ctypes.c_void_p), _np_ptr(te, np.int64)))


def ac_dev_exp_ticks(x_ptr: int, out_ptr: int, n: int) -> None:
    _check(_lib.ac_dev_exp_ticks(x_ptr, out_ptr, n))


def ac_dev_philox(seed: int, c_ptr: int, k_ptr: int, w2: int, out_ptr: int, n: int) -> None:
    _check(_lib.ac_dev_philox(seed & (2**64 - 1), c_ptr, k_ptr, w2, out_ptr, n))


def ac_run_blocked_static(rows: int, cols: int, beta: float, J: float, h: float, seed: int,
                          key_ptr: int, cnt_ptr: int, t_end: int, stream: int = 0) -> None:
    """Advance a lattice held in caller-owned device buffers without any allocation."""
    _check(_lib.ac_run_blocked_static(rows, cols, beta, J, h, seed & (2**64 - 1), key_ptr, cnt_ptr,
                                      int(t_end), stream))


def ac_frames_configure(sim: int, dt_ticks: int, K0: int, B: int) -> None:
    _check(_lib.ac_frames_configure(sim, int(dt_ticks), int(K0), int(B)))


def ac_run_until_frames(sim: int, t_end: int, fn=None, on_host: bool = True) -> None:
    """fn(K, ptr, n) is called for every completed frame; ptr is a host address (on_host) or a
    device address valid only during the call.  Exceptions raised by fn are re-raised here."""
    errors = []

    def _tramp(user, K, ptr, n):
        if errors:
            return
        try:
            fn(int(K), int(ptr), int(n))
        except BaseException as e:  # noqa: BLE001 -- re-raised after the C call returns
            errors.append(e)

    cb = FRAME_FN(_tramp) if fn is not None else FRAME_FN()
    status = _lib.ac_run_until_frames(sim, int(t_end), cb, None, 1 if on_host else 0)
    if errors:
        raise errors[0]
    _check(status)


def ac_frames_status(sim: int) -> tuple[int, int, int]:
    K, B, dt = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
    _check(_lib.ac_frames_status(sim, ctypes.byref(K), ctypes.byref(B), ctypes.byref(dt)))
    return K.value, B.value, dt.value


def ac_time_model(dims: int, n: int, law: int, seed: int, t_end: int, max_rounds: int, want_state: bool = False,
                  q: int = 1):
    """Time-only round model of Sec. 4 on the GPU (neighbourhood: Manhattan radius q): returns
    (advancing cells per round, final ticks or None, final counts or None, device milliseconds)."""
    en = np.zeros(max_rounds, dtype=np.uint64)
    rounds = ctypes.c_int32()
    ms = ctypes.c_double()
    N = n ** dims
    t = np.empty(N, dtype=np.int64) if want_state else None
    cnt = np.empty(N, dtype=np.uint32) if want_state else None
    _check(_lib.ac_time_model(int(dims), int(n), int(q), int(law), int(seed) & (2**64 - 1), int(t_end), int(max_rounds),
                              _np_ptr(en, np.uint64), ctypes.byref(rounds),
                              None if t is None else _np_ptr(t, np.int64),
                              None if cnt is None else _np_ptr(cnt, np.uint32), ctypes.byref(ms)))
    return en[:rounds.value].copy(), t, cnt, ms.value


# --------------------------------------------------------------- convenience
def life(rows: int, cols: int, seed: int = 0, density: float = 0.5, birth: int = AC_LIFE_CONWAY_BIRTH,
         survive: int = AC_LIFE_CONWAY_SURVIVE, init: int = 0, rounds: int = 6) -> "Sim":
    """A Sim handle holding an asynchronous Life-like automaton (alive = +1); density is the fraction
    of live cells of a random start (quantised to 32 bits)."""
    d = min(int(density * 2**32), 2**32 - 1) if density < 1.0 else 2**32 - 1
    h = ac_create_life(rows, cols, init, d, birth, survive, seed)
    sim = Sim(rows, cols, 0.0, 0.0, 0.0, seed, init=init, handle=h)
    sim.configure(AC_KERNEL_ROUND, 64, rounds, 0)
    return sim


def ising_q(rows: int, cols: int, beta: float, q: int, J: float = 1.0, h: float = 0.0, seed: int = 0,
            init: int = 0, rounds: int = 6) -> "Sim":
    """A Sim handle holding the Ising array on the q-th degree neighbourhood (q = 2, 3)."""
    hnd = ac_create_q(rows, cols, init, beta, J, h, q, seed)
    sim = Sim(rows, cols, beta, J, h, seed, init=init, handle=hnd)
    sim.configure(AC_KERNEL_ROUND, 64, rounds, 0)
    return sim


class Sim:
    """One lattice handle (owns its device memory; freed on close / GC)."""

    def __init__(self, rows: int, cols: int, beta: float, J: float = 1.0, h: float = 0.0, seed: int = 0,
                 init: int = AC_INIT_RANDOM, kernel: int | None = None, Lb: int | None = None,
                 rounds: int = 1, polls: int = 8, handle: int | None = None):
        self.rows, self.cols = int(rows), int(cols)
        self.beta, self.J, self.h, self.seed = float(beta), float(J), float(h), int(seed)
        self.handle = handle if handle is not None else ac_create(rows, cols, init, beta, J, h, seed)
        if kernel is not None or Lb is not None:
            self.configure(AC_KERNEL_BLOCKED if kernel is None else kernel, 64 if Lb is None else Lb,
                           rounds, polls)

    def configure(self, kernel: int, Lb: int, rounds: int = 1, polls: int = 8) -> "Sim":
        ac_configure(self.handle, kernel, Lb, rounds, polls)
        return self

    def set_stream(self, stream: int) -> None:
        ac_set_stream(self.handle, stream)

    def run_until(self, T: float) -> None:
        ac_run_until(self.handle, T)

    def run_until_ticks(self, t_end: int) -> None:
        ac_run_until_ticks(self.handle, t_end)

    def read_state(self):
        N = self.rows * self.cols
        s = np.empty(N, dtype=np.int8)
        t = np.empty(N, dtype=np.int64)
        n = np.empty(N, dtype=np.uint32)
        ac_read_state(self.handle, s, t, n)
        return s, t, n

    def load_state(self, s, t, n, t_done: int) -> None:
        ac_load_state(self.handle, np.ascontiguousarray(s, dtype=np.int8),
                      np.ascontiguousarray(t, dtype=np.int64), np.ascontiguousarray(n, dtype=np.uint32),
                      t_done)

    def stats(self) -> dict:
        return ac_stats(self.handle)

    def reset(self, seed: int, init: int = AC_INIT_RANDOM) -> None:
        ac_reset(self.handle, seed, init)
        self.seed = int(seed)

    def class_counts(self) -> np.ndarray:
        return ac_class_counts(self.handle)

    def set_rates(self, m) -> None:
        """Per-cell rates 2^20 / m[c] (None: all 1); re-initialises the handle at time 0."""
        ac_set_rates(self.handle, m)

    def set_option(self, option: int, value: int) -> None:
        ac_set_option(self.handle, option, value)

    def round_history(self) -> np.ndarray:
        return ac_round_history(self.handle)

    def configure_frames(self, dt_ticks: int, K0: int = 0, B: int = 4) -> None:
        """Snapshot frames K0, K0+1, ... at ticks K * dt_ticks, B frame slots (0 = off)."""
        ac_frames_configure(self.handle, dt_ticks, K0, B)

    def run_until_frames(self, t_end: int, on_frame=None) -> list:
        """Run to tick t_end.  Each completed frame K is passed as (K, int8 array of rows*cols
        spins) to on_frame, or collected and returned when on_frame is None."""
        got = []
        n_cells = self.rows * self.cols

        def _fn(K, ptr, n):
            assert n == n_cells
            frame = np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ctypes.c_int8)), shape=(n,)).copy()
            if on_frame is None:
                got.append((K, frame))
            else:
                on_frame(K, frame)

        ac_run_until_frames(self.handle, t_end, _fn, on_host=True)
        return got

    def frames_status(self) -> tuple[int, int, int]:
        return ac_frames_status(self.handle)

    def close(self) -> None:
        if self.handle:
            ac_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
