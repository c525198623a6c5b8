"""Plain serial CPU oracle for the Poisson-asynchronous Glauber cellular array.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline / reference leg of ``bench.py`` may import this package.
The library (``paper_cs_0502039_gb300``) never imports it, and nothing here
imports the library: the two implement the same definitions independently.

The arithmetic lives in ``ac_oracle.c`` (plain C99, compiled with gcc by
:func:`build`); this module only marshals numpy arrays through ctypes.

What it computes -- Lubachevsky, Sec. 1 (Poisson asynchrony, Glauber's
continuous-time Ising model), Sec. 2 Eqs. (1)-(2), Sec. 3 Eq. (5) and the
per-cell-stream remark after Fig. 3.6: all arrivals of all cells processed in
global (tick, cell index) order from a binary heap, each seeing the spins
just before it.  The spec readings R1-R7 are listed in ``ac_oracle.c``.

Pins (tests/test_oracle_*.py, all CPU):
  philox4x32_10   -- against triton's Philox4x32-10 (interpreter mode).
  exp_ticks       -- against binary64 -ln u (|err| <= 8 ticks), monotone,
                     ln 2 constant recomputed in exact decimal arithmetic.
  thresholds      -- detailed balance, beta = 0, spin-flip symmetry,
                     the appendix's x/(1+x) form.
  run             -- brute-force linear-scan simulator (bit-exact), exact
                     2x2 / 3x3 chain enumeration (stationary Boltzmann law,
                     transient P0 exp(QT)), Poisson(T) counts, beta = 0
                     closed form, Onsager energy and magnetisation.
  time_rounds     -- round-1 fraction 1/5, long-run fraction ~0.121 (Sec. 4).
  life_init, life_run -- brute-force linear scan, the rule on hand-built
                     neighbourhoods, still lifes, ticks equal to the Ising run's.
  gap, time_model -- laws: closed form, binary64 r^(1/8); brute-force rounds in
                     1, 2 and 3 dimensions; first-round fractions 1/3, 1/5, 1/7;
                     2D exponential equal to time_rounds; the paper's limits.
  frames          -- per-cell spin histories of the brute-force simulator read
                     at each frame time, including an arrival exactly at K dt.
  observables, checksum -- brute-force recomputation in numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ac_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libacoracle.so")

TICKS_PER_UNIT = 1 << 32
INIT_RANDOM, INIT_UP, INIT_DOWN = 0, 1, 2

_lib = None


def build(force: bool = False) -> str:
    """Compile ac_oracle.c into oracle/_build/libacoracle.so (gcc, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu99", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _bind(lib):
    """Declare the C signatures on a loaded oracle library."""
    P = ctypes.c_void_p
    lib.aco_philox4x32_10.argtypes = [P, P, P]
    lib.aco_philox4x32_10.restype = None
    lib.aco_exp_ticks.argtypes = [ctypes.c_uint32]
    lib.aco_exp_ticks.restype = ctypes.c_uint64
    lib.aco_thresholds.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, P]
    lib.aco_thresholds.restype = None
    lib.aco_init.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, P, P, P]
    lib.aco_init.restype = None
    lib.aco_run.argtypes = [ctypes.c_int32, ctypes.c_int32, P, ctypes.c_uint64, P, P, P, ctypes.c_int64]
    lib.aco_run.restype = ctypes.c_int64
    lib.aco_time_rounds.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, P, P,
                                    ctypes.c_int64, ctypes.c_int64, P]
    lib.aco_time_rounds.restype = ctypes.c_int64
    lib.aco_observables.argtypes = [ctypes.c_int32, ctypes.c_int32, P, P]
    lib.aco_observables.restype = None
    lib.aco_checksum.argtypes = [ctypes.c_int32, ctypes.c_int32, P, P, P]
    lib.aco_checksum.restype = ctypes.c_uint64
    lib.aco_exp_ticks_many.argtypes = [P, P, ctypes.c_int64]
    lib.aco_exp_ticks_many.restype = None
    lib.aco_philox_blocks.argtypes = [ctypes.c_uint64, P, P, ctypes.c_uint32, P, ctypes.c_int64]
    lib.aco_philox_blocks.restype = None
    lib.aco_class_counts.argtypes = [ctypes.c_int32, ctypes.c_int32, P, P]
    lib.aco_class_counts.restype = None
    lib.aco_thresholds_q.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int32, P]
    lib.aco_thresholds_q.restype = None
    lib.aco_run_q.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, ctypes.c_uint64, P, P, P,
                              ctypes.c_int64]
    lib.aco_run_q.restype = ctypes.c_int64
    lib.aco_rated_gap.argtypes = [ctypes.c_uint64, ctypes.c_uint32]
    lib.aco_rated_gap.restype = ctypes.c_uint64
    lib.aco_init_rated.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, P, P, P, P]
    lib.aco_init_rated.restype = None
    lib.aco_run_rated.argtypes = [ctypes.c_int32, ctypes.c_int32, P, ctypes.c_uint64, P, P, P, P, ctypes.c_int64]
    lib.aco_run_rated.restype = ctypes.c_int64
    lib.aco_life_init.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32,
                                  ctypes.c_uint64, P, P, P]
    lib.aco_life_init.restype = None
    lib.aco_life_run.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint32,
                                 ctypes.c_uint64, P, P, P, ctypes.c_int64]
    lib.aco_life_run.restype = ctypes.c_int64
    lib.aco_gap.argtypes = [ctypes.c_int32, ctypes.c_uint32]
    lib.aco_gap.restype = ctypes.c_uint64
    lib.aco_time_model.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, P, P, P]
    lib.aco_time_model.restype = ctypes.c_int64
    return lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one 4-word counter under a 2-word key -> uint32[4]."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.aco_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def exp_ticks(x: int) -> int:
    """Integer exponential gap (ticks) for a 32-bit uniform word x."""
    return int(_load().aco_exp_ticks(ctypes.c_uint32(int(x) & 0xFFFFFFFF)))


def exp_ticks_many(xs) -> np.ndarray:
    """exp_ticks over an array of 32-bit words -> uint64 array."""
    x = np.ascontiguousarray(xs, dtype=np.uint32)
    out = np.zeros(x.shape, dtype=np.uint64)
    _load().aco_exp_ticks_many(_ptr(x), _ptr(out), x.size)
    return out


def philox_blocks(seed: int, cells, ks, w2: int = 0) -> np.ndarray:
    """Philox({c, k, w2, 0}) under key (seed lo, seed hi) for arrays c, k -> uint32[n, 4]."""
    c = np.ascontiguousarray(cells, dtype=np.uint32)
    k = np.ascontiguousarray(np.broadcast_to(ks, c.shape), dtype=np.uint32)
    out = np.zeros((c.size, 4), dtype=np.uint32)
    _load().aco_philox_blocks(int(seed) & (2**64 - 1), _ptr(c), _ptr(k), int(w2), _ptr(out), c.size)
    return out


def thresholds(beta: float, J: float = 1.0, h: float = 0.0) -> np.ndarray:
    """uint32[10] flip thresholds, index j + 5*(s>0), j = number of up neighbours."""
    out = np.zeros(10, dtype=np.uint32)
    _load().aco_thresholds(float(beta), float(J), float(h), _ptr(out))
    return out


class State:
    """A lattice state: spins int8, next-arrival ticks int64, event counts uint32."""

    def __init__(self, rows: int, cols: int, s: np.ndarray, t: np.ndarray, n: np.ndarray):
        self.rows, self.cols = int(rows), int(cols)
        self.s, self.t, self.n = s, t, n

    def copy(self) -> "State":
        return State(self.rows, self.cols, self.s.copy(), self.t.copy(), self.n.copy())


def init(rows: int, cols: int, init_mode: int, seed: int) -> State:
    """Initial state from the seed (readings R3, R4)."""
    if rows < 2 or cols < 2:
        raise ValueError("rows and cols must be >= 2")
    N = rows * cols
    s = np.zeros(N, dtype=np.int8)
    t = np.zeros(N, dtype=np.int64)
    n = np.zeros(N, dtype=np.uint32)
    _load().aco_init(rows, cols, int(init_mode), int(seed) & (2**64 - 1), _ptr(s), _ptr(t), _ptr(n))
    return State(rows, cols, s, t, n)


def run(state: State, thr: np.ndarray, seed: int, t_end: int) -> int:
    """Advance ``state`` in place until every tick >= t_end; returns events committed."""
    thr = np.ascontiguousarray(thr, dtype=np.uint32)
    ev = _load().aco_run(state.rows, state.cols, _ptr(thr), int(seed) & (2**64 - 1),
                         _ptr(state.s), _ptr(state.t), _ptr(state.n), int(t_end))
    if ev < 0:
        raise MemoryError("oracle heap allocation failed")
    return int(ev)


def frames(state: State, thr: np.ndarray, seed: int, dt_ticks: int, K0: int, count: int) -> np.ndarray:
    """Snapshot frames K0 .. K0+count-1 (Sec. 3, "Generating the output", Fig. 3.7).

    Frame K is every cell's spin after all of its arrivals with tick <= K * dt_ticks:
    the figure stores a subarray's image before it processes the first event later
    than K dt (reading R10).  With ``run``'s strict end (tick < t_end) that is the
    state after ``run(.., K * dt_ticks + 1)``.  ``state`` must not be past frame K0
    (it was last run to a t_end <= K0 * dt_ticks + 1).  Advances ``state`` in place
    to the last frame; returns an int8 array of shape (count, rows * cols)."""
    out = np.zeros((count, state.rows * state.cols), dtype=np.int8)
    for i in range(count):
        run(state, thr, seed, (K0 + i) * dt_ticks + 1)
        out[i] = state.s
    return out


def simulate(rows: int, cols: int, beta: float, J: float, h: float, seed: int, T: float,
             init_mode: int = INIT_RANDOM) -> State:
    """Fresh lattice run to time T (t_end = T * 2^32 ticks, rounded down)."""
    st = init(rows, cols, init_mode, seed)
    run(st, thresholds(beta, J, h), seed, int(T * TICKS_PER_UNIT))
    return st


def time_rounds(state: State, seed: int, t_end: int, max_rounds: int = 1 << 20):
    """Time-only synchronous rounds (Sec. 4 model of Fig. 3.2); advances state.t/.n in place.

    Returns int64 array with the number of advancing cells in each round.
    """
    buf = np.zeros(max_rounds, dtype=np.int64)
    r = _load().aco_time_rounds(state.rows, state.cols, int(seed) & (2**64 - 1), _ptr(state.t),
                                _ptr(state.n), int(t_end), int(max_rounds), _ptr(buf))
    if r < 0:
        raise MemoryError("oracle allocation failed")
    return buf[:min(r, max_rounds)].copy()


def thresholds_q(beta: float, J: float, h: float, q: int) -> np.ndarray:
    """Heat-bath table of the q-th degree neighbourhood (reading R14): index j + (M+1)(s>0),
    M = 2q(q+1) neighbours, j of them up."""
    M = 2 * q * (q + 1)
    out = np.zeros(2 * (M + 1), dtype=np.uint32)
    _load().aco_thresholds_q(float(beta), float(J), float(h), int(q), _ptr(out))
    return out


def run_q(state: State, q: int, thr: np.ndarray, seed: int, t_end: int) -> int:
    """As run(), for the Ising array on the q-th degree neighbourhood (every cell within Manhattan
    distance q); thr from thresholds_q."""
    if state.rows < 2 * q + 1 or state.cols < 2 * q + 1:
        raise ValueError("rows and cols must be >= 2q + 1")
    thr = np.ascontiguousarray(thr, dtype=np.uint32)
    ev = _load().aco_run_q(state.rows, state.cols, int(q), _ptr(thr), int(seed) & (2**64 - 1), _ptr(state.s),
                           _ptr(state.t), _ptr(state.n), int(t_end))
    if ev < 0:
        raise MemoryError("oracle heap allocation failed")
    return int(ev)


RATE_ONE = 1 << 20      # multiplier m of rate p = 2^20 / m


def rated_gap(e: int, m: int) -> int:
    """Gap of a cell with rate 2^20 / m for the rate-1 gap e (reading R13)."""
    return int(_load().aco_rated_gap(int(e), int(m) & 0xFFFFFFFF))


def init_rated(rows: int, cols: int, init_mode: int, seed: int, m) -> State:
    """Initial state with per-cell rates 2^20 / m[c] (first arrivals scaled, reading R13)."""
    st = init(rows, cols, init_mode, seed)
    m = np.ascontiguousarray(m, dtype=np.uint32)
    _load().aco_init_rated(rows, cols, int(init_mode), int(seed) & (2**64 - 1), _ptr(m), _ptr(st.s), _ptr(st.t),
                           _ptr(st.n))
    return st


def run_rated(state: State, thr: np.ndarray, seed: int, m, t_end: int) -> int:
    """As run(), with every gap scaled for the cell's rate 2^20 / m[c]."""
    thr = np.ascontiguousarray(thr, dtype=np.uint32)
    m = np.ascontiguousarray(m, dtype=np.uint32)
    ev = _load().aco_run_rated(state.rows, state.cols, _ptr(thr), int(seed) & (2**64 - 1), _ptr(m), _ptr(state.s),
                               _ptr(state.t), _ptr(state.n), int(t_end))
    if ev < 0:
        raise MemoryError("oracle heap allocation failed")
    return int(ev)


CONWAY_BIRTH, CONWAY_SURVIVE = 1 << 3, (1 << 2) | (1 << 3)


def life_init(rows: int, cols: int, init_mode: int, density: int, seed: int) -> State:
    """Initial Life state (reading R12): alive (+1) iff I(c).x < density for init 0, all alive for 1,
    all dead for 2; first arrivals as for the Ising array."""
    if rows < 3 or cols < 3:
        raise ValueError("rows and cols must be >= 3")
    N = rows * cols
    s = np.zeros(N, dtype=np.int8)
    t = np.zeros(N, dtype=np.int64)
    n = np.zeros(N, dtype=np.uint32)
    _load().aco_life_init(rows, cols, int(init_mode), int(density) & 0xFFFFFFFF, int(seed) & (2**64 - 1),
                          _ptr(s), _ptr(t), _ptr(n))
    return State(rows, cols, s, t, n)


def life_run(state: State, birth: int, survive: int, seed: int, t_end: int) -> int:
    """Advance a Life state in place: every arrival with tick < t_end, in (tick, index) order, sets the
    cell to bit k of `survive` (alive) or `birth` (dead), k = live Moore neighbours just before it."""
    ev = _load().aco_life_run(state.rows, state.cols, int(birth), int(survive), int(seed) & (2**64 - 1),
                              _ptr(state.s), _ptr(state.t), _ptr(state.n), int(t_end))
    if ev < 0:
        raise MemoryError("oracle heap allocation failed")
    return int(ev)


LAW_EXP, LAW_UNIFORM, LAW_ROOT8 = 0, 1, 2


def gap(law: int, x: int) -> int:
    """Increment in ticks for the 32-bit word x under law 0 (exponential), 1 (uniform on (0, 1])
    or 2 (r^(1/8)) of the time-only model (reading R11)."""
    return int(_load().aco_gap(int(law), int(x) & 0xFFFFFFFF))


def time_model(dims: int, n: int, law: int, seed: int, t_end: int, max_rounds: int, q: int = 1):
    """Time-only round model of Sec. 4 on an n-cell circle (dims 1), n x n torus (2) or n^3
    periodic array (3), with the q-th degree neighbourhood of Sec. 3 (every cell within
    Manhattan distance q; q = 1 is the nearest neighbours): returns (advancing cells per
    round, final ticks, final counts)."""
    N = n ** dims
    en = np.zeros(max(1, max_rounds), dtype=np.int64)
    t = np.zeros(N, dtype=np.int64)
    cnt = np.zeros(N, dtype=np.uint32)
    r = _load().aco_time_model(int(dims), int(n), int(q), int(law), int(seed) & (2**64 - 1), int(t_end),
                               int(max_rounds), _ptr(en), _ptr(t), _ptr(cnt))
    if r == -1:
        raise MemoryError("oracle allocation failed")
    if r < 0:
        raise ValueError("dims must be 1..3, n >= 2, law 0..2, q in 1..8 with n >= 2q+1")
    return en[:r].copy(), t, cnt


def class_counts(state: State) -> np.ndarray:
    """Cells per BKL class (Sec. 3): index j + 5 (s > 0), j = up neighbours, as in the table."""
    out = np.zeros(10, dtype=np.int64)
    _load().aco_class_counts(state.rows, state.cols, _ptr(state.s), _ptr(out))
    return out


def observables(state: State):
    """(sum of spins, sum over right+down bonds of s s')."""
    out = np.zeros(2, dtype=np.int64)
    _load().aco_observables(state.rows, state.cols, _ptr(state.s), _ptr(out))
    return int(out[0]), int(out[1])


def checksum(state: State) -> int:
    """Order-independent 64-bit fingerprint of (s, t, n)."""
    return int(_load().aco_checksum(state.rows, state.cols, _ptr(state.s), _ptr(state.t),
                                    _ptr(state.n)))
