"""ctypes declarations mirroring include/ridfa.h, with the same function names."""

import ctypes
import os
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libridfa.so")

if not os.path.exists(_LIB_PATH):
    raise ImportError(
        f"libridfa.so is not built ({_LIB_PATH}); run `python paper_2412_14975_gb300/build_lib.py` "
        "(the recognizer has no CPU fallback)")

_lib = ctypes.CDLL(_LIB_PATH)

RIDFA_UNDEF = 0xFFFF
RIDFA_MAX_STATES = 65534
RIDFA_MAX_SLOTS = 256
RIDFA_NOALLOC_SCRATCH_BYTES = 4 << 20

_c = ctypes
_vp = _c.c_void_p
_u32 = _c.c_uint32


class CompileOpts(_c.Structure):
    _fields_ = [("minimize_interface", _u32), ("build_dfa", _u32), ("max_states", _u32)]


class Info(_c.Structure):
    _fields_ = [("n_nfa", _u32), ("n_states", _u32), ("k", _u32), ("n_classes", _u32),
                ("n_dfa_states", _u32), ("q0_slot", _u32), ("table_bytes", _c.c_uint64),
                ("dfa_table_bytes", _c.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Tuning(_c.Structure):
    _fields_ = [("piece_len", _u32), ("block_threads", _u32), ("probe_interval", _u32),
                ("grid_blocks", _u32), ("profile", _u32), ("table_mode", _u32),
                ("text_path", _u32), ("lookback_cap", _u32)]


def _decl(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_decl("ridfa_compile", _c.c_int, [_c.c_char_p, _c.c_size_t, _c.POINTER(CompileOpts), _c.POINTER(_vp)])
_decl("ridfa_free", None, [_vp])
_decl("ridfa_program_info", _c.c_int, [_vp, _c.POINTER(Info)])
_decl("ridfa_state_set", _c.c_int, [_vp, _u32, _vp, _u32, _c.POINTER(_u32)])
_decl("ridfa_slots", _c.c_int, [_vp, _vp])
_decl("ridfa_delegates", _c.c_int, [_vp, _vp])
_decl("ridfa_export_tables", _c.c_int, [_vp, _c.c_int, _vp, _vp, _vp])
for _n in ("ridfa_recognize", "ridfa_recognize_async", "ridfa_recognize_dfa", "ridfa_recognize_dfa_async"):
    _decl(_n, _c.c_int, [_vp, _vp, _c.c_size_t, _u32, _c.POINTER(Tuning), _vp, _vp, _vp])
_decl("ridfa_recognize_host", _c.c_int, [_vp, _vp, _c.c_size_t, _u32, _c.POINTER(Tuning), _vp, _vp, _vp])
_decl("ridfa_last_status", _c.c_int, [_vp, _vp])
_decl("ridfa_check_bounded_wait", _c.c_int, [_u32, _c.c_int, _vp])
_decl("ridfa_recognize_noalloc", _c.c_int, [_vp, _vp, _c.c_size_t, _u32, _vp, _vp, _vp])
_decl("ridfa_bench_smem_gather", _c.c_int, [_u32, _c.POINTER(_c.c_double), _c.POINTER(_c.c_double)])
_decl("ridfa_bench_hbm_read", _c.c_int, [_vp, _c.c_size_t, _c.POINTER(_c.c_double), _c.POINTER(_c.c_double)])
_decl("ridfa_strerror", _c.c_char_p, [_c.c_int])
_decl("ridfa_last_timings", _c.c_int, [_vp, _c.POINTER(_c.c_float), _c.POINTER(_c.c_float)])


class PlanReport(_c.Structure):
    _fields_ = [("table_mode", _u32), ("text_path", _u32), ("lane_copies", _u32),
                ("block_threads", _u32), ("grid_blocks", _u32), ("pieces", _u32)]


_decl("ridfa_last_plan", _c.c_int, [_vp, _c.POINTER(PlanReport)])


class RidfaError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {ridfa_strerror(code)} ({code})")


def lib_path():
    return _LIB_PATH


def ridfa_strerror(code):
    return _lib.ridfa_strerror(int(code)).decode()


def _check(code, where):
    if code != 0:
        raise RidfaError(code, where)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take a device address of {type(x)}")


def _stream(s):
    if s is None:
        torch = sys.modules.get("torch")
        if torch is not None and torch.cuda.is_available() and torch.cuda.is_initialized():
            return torch.cuda.current_stream().cuda_stream
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


class Program:
    """Owns one ridfa_program*; freed with ridfa_free when collected or closed."""

    def __init__(self, handle, re_src):
        self.handle = handle
        self.re = re_src
        self._info = ridfa_program_info(self)

    @property
    def info(self):
        return self._info

    def close(self):
        if self.handle:
            ridfa_free(self)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        if not self.handle:
            raise ValueError("program is closed")
        return self.handle


def ridfa_compile(re_src, minimize_interface=True, build_dfa=True, max_states=0):
    raw = re_src.encode("latin-1") if isinstance(re_src, str) else bytes(re_src)
    opts = CompileOpts(int(bool(minimize_interface)), int(bool(build_dfa)), int(max_states))
    h = _vp()
    _check(_lib.ridfa_compile(raw, len(raw), _c.byref(opts), _c.byref(h)), "ridfa_compile")
    return Program(h.value, re_src)


def ridfa_free(prog):
    _lib.ridfa_free(prog.handle)


def ridfa_program_info(prog):
    info = Info()
    _check(_lib.ridfa_program_info(_vp(prog.handle), _c.byref(info)), "ridfa_program_info")
    return info.as_dict()


def ridfa_state_set(prog, state):
    n = _u32()
    _lib.ridfa_state_set(prog, int(state), None, 0, _c.byref(n))
    out = np.zeros(max(1, n.value), dtype=np.uint32)
    _check(_lib.ridfa_state_set(prog, int(state), out.ctypes.data, out.size, _c.byref(n)),
           "ridfa_state_set")
    return out[:n.value].copy()


def ridfa_slots(prog):
    out = np.zeros(max(1, prog.info["k"]), dtype=np.uint32)
    _check(_lib.ridfa_slots(prog, out.ctypes.data), "ridfa_slots")
    return out[:prog.info["k"]]


def ridfa_delegates(prog):
    out = np.zeros(prog.info["n_nfa"], dtype=np.uint32)
    _check(_lib.ridfa_delegates(prog, out.ctypes.data), "ridfa_delegates")
    return out


def ridfa_export_tables(prog, which=0):
    """(trans [(n+1), C] uint16, classmap [256] uint8, final [n] uint8) of the RI-DFA (0) or
    the minimal DFA (1)."""
    info = prog.info
    n = info["n_states"] if which == 0 else info["n_dfa_states"]
    if which == 1 and n == 0:
        raise RidfaError(-10, "ridfa_export_tables")
    trans = np.zeros((n + 1) * info["n_classes"], dtype=np.uint16)
    cmap = np.zeros(256, dtype=np.uint8)
    fin = np.zeros(max(1, n), dtype=np.uint8)
    _check(_lib.ridfa_export_tables(prog, int(which), trans.ctypes.data, cmap.ctypes.data,
                                    fin.ctypes.data), "ridfa_export_tables")
    return trans.reshape(n + 1, info["n_classes"]), cmap, fin[:n]


def _tuning(t):
    if t is None:
        return None
    if isinstance(t, Tuning):
        return _c.byref(t)
    return _c.byref(Tuning(t.get("piece_len", 0), t.get("block_threads", 0),
                           t.get("probe_interval", 0), t.get("grid_blocks", 0),
                           t.get("profile", 0), t.get("table_mode", 0), t.get("text_path", 0),
                           t.get("lookback_cap", 0)))


def _recognize_sync(fn, name, prog, text, length, n_chunks, tuning, maps, stream):
    acc = _c.c_uint8(0)
    _check(fn(prog, _ptr(text), int(length), int(n_chunks), _tuning(tuning),
              _c.addressof(acc), _ptr(maps), _stream(stream)), name)
    return bool(acc.value)


def _recognize_async(fn, name, prog, text, length, n_chunks, d_accept, tuning, maps, stream):
    _check(fn(prog, _ptr(text), int(length), int(n_chunks), _tuning(tuning),
              _ptr(d_accept), _ptr(maps), _stream(stream)), name)


def ridfa_recognize(prog, d_text, length, n_chunks, tuning=None, d_chunk_maps=None, stream=None):
    """Accept bit of the text (device buffer) by the RID; synchronises the stream."""
    return _recognize_sync(_lib.ridfa_recognize, "ridfa_recognize", prog, d_text, length,
                           n_chunks, tuning, d_chunk_maps, stream)


def ridfa_recognize_host(prog, h_text, length, n_chunks, d_staging, tuning=None, stream=None):
    """Accept bit of a text in host memory (a page-locked CPU tensor, a numpy array or a bytes-like
    object), copied by the library into the device buffer d_staging and recognized there;
    synchronises the stream."""
    if isinstance(h_text, (bytes, bytearray, memoryview)):
        h_text = np.frombuffer(h_text, dtype=np.uint8)
    acc = _c.c_uint8(0)
    _check(_lib.ridfa_recognize_host(prog, _ptr(h_text), int(length), int(n_chunks), _tuning(tuning),
                                     _ptr(d_staging), _c.addressof(acc), _stream(stream)),
           "ridfa_recognize_host")
    return bool(acc.value)


def ridfa_check_bounded_wait(limit, arrive, stream=None):
    """Status code of one bounded device wait: RIDFA_OK (0) when the phase completed, -7
    (E_TIMEOUT) when `limit` polls ran out (arrive=False: nothing ever arrives)."""
    return int(_lib.ridfa_check_bounded_wait(int(limit), 1 if arrive else 0, _stream(stream)))


def ridfa_recognize_async(prog, d_text, length, n_chunks, d_accept, tuning=None,
                          d_chunk_maps=None, stream=None):
    _recognize_async(_lib.ridfa_recognize_async, "ridfa_recognize_async", prog, d_text, length,
                     n_chunks, d_accept, tuning, d_chunk_maps, stream)


def ridfa_recognize_dfa(prog, d_text, length, n_chunks, tuning=None, d_chunk_maps=None, stream=None):
    """Accept bit by the all-states minimal-DFA comparator; synchronises the stream."""
    return _recognize_sync(_lib.ridfa_recognize_dfa, "ridfa_recognize_dfa", prog, d_text, length,
                           n_chunks, tuning, d_chunk_maps, stream)


def ridfa_recognize_dfa_async(prog, d_text, length, n_chunks, d_accept, tuning=None,
                              d_chunk_maps=None, stream=None):
    _recognize_async(_lib.ridfa_recognize_dfa_async, "ridfa_recognize_dfa_async", prog, d_text,
                     length, n_chunks, d_accept, tuning, d_chunk_maps, stream)


_decl("ridfa_recognize_nfa", _c.c_int, [_vp, _vp, _c.c_size_t, _u32, _c.POINTER(_c.c_uint8), _vp, _vp])


def ridfa_recognize_nfa(prog, d_text, length, n_chunks, d_sets=None, stream=None):
    """Accept bit by the NFA variant of the classic algorithm (every position-NFA state a start
    state, sets simulated per start); d_sets optionally receives the chunk relations as
    [n_chunks][n_nfa][ceil(n_nfa / 32)] uint32 bitsets.  Synchronises the stream."""
    acc = _c.c_uint8(0)
    _check(_lib.ridfa_recognize_nfa(prog, _ptr(d_text) if length else None, int(length), int(n_chunks),
                                    _c.byref(acc), _ptr(d_sets) if d_sets is not None else None, _stream(stream)),
           "ridfa_recognize_nfa")
    return bool(acc.value)


def ridfa_last_status(prog, stream=None):
    code = _lib.ridfa_last_status(prog, _stream(stream))
    return code


def ridfa_last_plan(prog):
    """The reach plan of the program's last recognition on the current device: dict with
    table_mode, text_path, lane_copies, block_threads, grid_blocks, pieces."""
    out = PlanReport()
    _check(_lib.ridfa_last_plan(prog, _c.byref(out)), "ridfa_last_plan")
    return {f: getattr(out, f) for f, _ in out._fields_}


def ridfa_last_timings(prog):
    """(reach_ms, join_ms) of the last call made with tuning profile=1."""
    a, b = _c.c_float(), _c.c_float()
    _check(_lib.ridfa_last_timings(prog, _c.byref(a), _c.byref(b)), "ridfa_last_timings")
    return a.value, b.value


def ridfa_recognize_noalloc(prog, d_text, length, n_chunks, d_accept, d_chunk_maps, stream=None):
    """RID path that allocates no device memory: tables and scratch live in the library's fixed
    RIDFA_NOALLOC_SCRATCH_BYTES device array; d_chunk_maps (n_chunks * k uint16) is required.
    Asynchronous on `stream`; overlapping calls share the array and must be serialised."""
    _check(_lib.ridfa_recognize_noalloc(prog, _ptr(d_text), int(length), int(n_chunks),
                                        _ptr(d_accept), _ptr(d_chunk_maps), _stream(stream)),
           "ridfa_recognize_noalloc")


def ridfa_bench_smem_gather(iters=1 << 16):
    """Text bytes per second of the converged step alone (two lane-private gathers per byte)."""
    r, ms = _c.c_double(), _c.c_double()
    _check(_lib.ridfa_bench_smem_gather(int(iters), _c.byref(r), _c.byref(ms)), "ridfa_bench_smem_gather")
    return r.value


def ridfa_bench_hbm_read(d_buf, nbytes):
    """Streaming-read bytes per second over a 16-byte-aligned device buffer."""
    r, ms = _c.c_double(), _c.c_double()
    _check(_lib.ridfa_bench_hbm_read(_ptr(d_buf), int(nbytes), _c.byref(r), _c.byref(ms)), "ridfa_bench_hbm_read")
    return r.value


# ---------------------------------------------------------------------------------- batches
class BatchItem(_c.Structure):
    _fields_ = [("d_text", _vp), ("len", _c.c_uint64), ("prog", _u32), ("n_chunks", _u32)]


class BatchOpts(_c.Structure):
    _fields_ = [("chunk_len", _u32), ("no_graph", _u32), ("block_warps", _u32), ("set_mode", _u32)]


class BatchStats(_c.Structure):
    _fields_ = [("total_bytes", _c.c_uint64), ("total_chunks", _c.c_uint64), ("n_programs", _u32),
                ("n_launches", _u32), ("n_tasks", _u32), ("n_segments", _u32), ("chunk_len", _u32),
                ("block_warps", _u32), ("set_mode", _u32), ("graph", _u32), ("device_bytes", _c.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_decl("ridfa_batch_create", _c.c_int, [_c.POINTER(_vp), _u32, _c.POINTER(BatchItem), _u32, _vp,
                                       _c.POINTER(BatchOpts), _c.POINTER(_vp)])
_decl("ridfa_batch_run", _c.c_int, [_vp, _vp])
_decl("ridfa_batch_get_stats", _c.c_int, [_vp, _c.POINTER(BatchStats)])
_decl("ridfa_batch_free", None, [_vp])
_decl("ridfa_recognize_batch", _c.c_int, [_c.POINTER(_vp), _u32, _c.POINTER(BatchItem), _u32, _vp, _vp])


def _batch_arrays(progs, items):
    parr = (_vp * len(progs))(*[p.handle for p in progs])
    iarr = (BatchItem * len(items))()
    for i, (text, length, prog, n_chunks) in enumerate(items):
        iarr[i] = BatchItem(_ptr(text) if length else None, int(length), int(prog), int(n_chunks))
    return parr, iarr


class Batch:
    """Owns one ridfa_batch*; keeps its programs alive."""

    def __init__(self, handle, progs):
        self.handle = handle
        self.progs = list(progs)

    def close(self):
        if self.handle:
            _lib.ridfa_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        if not self.handle:
            raise ValueError("batch is closed")
        return self.handle


def ridfa_batch_create(progs, items, d_accept, chunk_len=0, no_graph=False, block_warps=0, set_mode=0):
    """items: list of (device text, length, program index, n_chunks or 0)."""
    parr, iarr = _batch_arrays(progs, items)
    opts = BatchOpts(int(chunk_len), int(bool(no_graph)), int(block_warps), int(set_mode))
    h = _vp()
    _check(_lib.ridfa_batch_create(parr, len(progs), iarr, len(items), _ptr(d_accept), _c.byref(opts),
                                   _c.byref(h)), "ridfa_batch_create")
    return Batch(h.value, progs)


def ridfa_batch_run(batch, stream=None):
    _check(_lib.ridfa_batch_run(batch, _stream(stream)), "ridfa_batch_run")


def ridfa_batch_get_stats(batch):
    st = BatchStats()
    _check(_lib.ridfa_batch_get_stats(batch, _c.byref(st)), "ridfa_batch_get_stats")
    return st.as_dict()


def ridfa_batch_free(batch):
    batch.close()


def ridfa_recognize_batch(progs, items, d_accept, stream=None):
    parr, iarr = _batch_arrays(progs, items)
    _check(_lib.ridfa_recognize_batch(parr, len(progs), iarr, len(items), _ptr(d_accept), _stream(stream)),
           "ridfa_recognize_batch")


# ---------------------------------------------------------------------------------- serving
RIDFA_SUBMIT_DEVICE_TEXT = 1


class ServerOpts(_c.Structure):
    _fields_ = [("device", _c.c_int32), ("n_streams", _u32), ("arena_bytes", _c.c_uint64),
                ("max_requests", _u32), ("max_batch_requests", _u32), ("max_batch_bytes", _c.c_uint64),
                ("chunk_len", _u32), ("reserved", _u32), ("device_budget", _c.c_uint64)]


class Result(_c.Structure):
    _fields_ = [("req_id", _c.c_uint64), ("status", _c.c_int32), ("accept", _u32),
                ("latency_us", _c.c_double)]


class ServerStats(_c.Structure):
    _fields_ = [("submitted", _c.c_uint64), ("completed", _c.c_uint64), ("rejected", _c.c_uint64),
                ("batches", _c.c_uint64), ("bytes", _c.c_uint64), ("max_batch", _u32),
                ("n_programs", _u32), ("device_bytes", _c.c_uint64), ("table_bytes", _c.c_uint64),
                ("budget_used", _c.c_uint64), ("budget_peak", _c.c_uint64), ("batch_hist", _u32 * 16)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "batch_hist"}
        d["batch_hist"] = list(self.batch_hist)
        return d


class LoadgenRecord(_c.Structure):
    _fields_ = [("text", _u32), ("status", _c.c_int32), ("accept", _u32), ("busy_retries", _u32),
                ("latency_us", _c.c_double), ("server_us", _c.c_double)]


_decl("ridfa_server_create", _c.c_int, [_c.POINTER(ServerOpts), _c.POINTER(_vp)])
_decl("ridfa_server_add_program", _c.c_int, [_vp, _vp, _c.POINTER(_u32)])
_decl("ridfa_server_submit", _c.c_int, [_vp, _u32, _vp, _c.c_uint64, _u32, _c.POINTER(_c.c_uint64)])
_decl("ridfa_server_poll", _c.c_int, [_vp, _c.POINTER(Result), _u32, _c.POINTER(_u32), _u32])
_decl("ridfa_server_drain", _c.c_int, [_vp, _u32])
_decl("ridfa_server_get_stats", _c.c_int, [_vp, _c.POINTER(ServerStats)])
_decl("ridfa_server_destroy", None, [_vp])
_decl("ridfa_bench_served_poisson", _c.c_int, [_vp, _vp, _vp, _vp, _u32, _c.c_double, _c.c_double,
                                                _c.c_uint64, _c.POINTER(LoadgenRecord), _u32,
                                                _c.POINTER(_u32), _c.POINTER(_c.c_double), _u32])


class Server:
    """Owns one ridfa_server*; keeps its programs alive.

    submit() takes a host text (bytes, bytearray or a contiguous uint8 numpy array), copied into
    the server's arena before it returns, or a CUDA uint8 tensor / device address with
    device=True (read in place: keep it alive until its result is polled)."""

    def __init__(self, device=-1, n_streams=0, arena_bytes=0, max_requests=0, max_batch_requests=0,
                 max_batch_bytes=0, chunk_len=0, device_budget=0):
        opts = ServerOpts(int(device), int(n_streams), int(arena_bytes), int(max_requests),
                          int(max_batch_requests), int(max_batch_bytes), int(chunk_len), 0,
                          int(device_budget))
        h = _vp()
        _check(_lib.ridfa_server_create(_c.byref(opts), _c.byref(h)), "ridfa_server_create")
        self.handle = h.value
        self.progs = []
        self._res = (Result * 4096)()

    def add_program(self, prog):
        slot = _u32()
        _check(_lib.ridfa_server_add_program(self, prog, _c.byref(slot)), "ridfa_server_add_program")
        self.progs.append(prog)
        return slot.value

    def submit(self, prog_slot, text, length=None, device=False):
        """Returns the request id; raises RidfaError (code -8, E_BUSY) when admission is refused."""
        if device:
            ptr = _ptr(text)
            n = int(length if length is not None else text.numel())
            flags = RIDFA_SUBMIT_DEVICE_TEXT
        else:
            if isinstance(text, (bytes, bytearray)):
                buf = np.frombuffer(text, dtype=np.uint8)
            else:
                buf = np.ascontiguousarray(text, dtype=np.uint8)
            n = int(length if length is not None else buf.size)
            ptr = buf.ctypes.data if n else None
            flags = 0
        rid = _c.c_uint64()
        _check(_lib.ridfa_server_submit(self, int(prog_slot), ptr, n, flags, _c.byref(rid)), "ridfa_server_submit")
        return rid.value

    def try_submit(self, prog_slot, text, length=None, device=False):
        """As submit(), but returns None instead of raising when the server is busy."""
        try:
            return self.submit(prog_slot, text, length, device)
        except RidfaError as e:
            if e.code == -8:
                return None
            raise

    def poll(self, max_results=4096, wait_us=0):
        """List of (req_id, status, accept, latency_us)."""
        n = _u32()
        m = min(int(max_results), len(self._res))
        _check(_lib.ridfa_server_poll(self, self._res, m, _c.byref(n), int(wait_us)), "ridfa_server_poll")
        return [(r.req_id, r.status, bool(r.accept), r.latency_us) for r in self._res[:n.value]]

    def drain(self, timeout_ms=60_000):
        _check(_lib.ridfa_server_drain(self, int(timeout_ms)), "ridfa_server_drain")

    def bench_poisson(self, prog_slots, texts, rate_rps, seconds, seed, device_texts=None):
        """ridfa_bench_served_poisson over a pool of host texts (contiguous uint8 numpy arrays,
        one program slot each), or of device texts (device_texts: (pointer, length) pairs, read in
        place).  Returns (records as a structured numpy array, wall seconds)."""
        if device_texts is not None:
            n = len(device_texts)
            bufs = []
            ptrs = (_vp * n)(*[int(p) if ln else None for p, ln in device_texts])
            lens = (_c.c_uint64 * n)(*[int(ln) for _, ln in device_texts])
            flags = RIDFA_SUBMIT_DEVICE_TEXT
        else:
            n = len(texts)
            bufs = [np.ascontiguousarray(t, dtype=np.uint8) for t in texts]
            ptrs = (_vp * n)(*[b.ctypes.data if b.size else None for b in bufs])
            lens = (_c.c_uint64 * n)(*[int(b.size) for b in bufs])
            flags = 0
        slots = (_u32 * n)(*[int(p) for p in prog_slots])
        cap = int(rate_rps * seconds * 1.5) + 1000
        recs = (LoadgenRecord * cap)()
        n_out, wall = _u32(), _c.c_double()
        _check(_lib.ridfa_bench_served_poisson(self, slots, ptrs, lens, n, float(rate_rps), float(seconds),
                                               int(seed), recs, cap, _c.byref(n_out), _c.byref(wall), flags),
               "ridfa_bench_served_poisson")
        out = np.frombuffer(recs, dtype=np.dtype([("text", "<u4"), ("status", "<i4"), ("accept", "<u4"),
                                                  ("busy_retries", "<u4"), ("latency_us", "<f8"),
                                                  ("server_us", "<f8")]), count=n_out.value).copy()
        del bufs
        return out, wall.value

    def stats(self):
        st = ServerStats()
        _check(_lib.ridfa_server_get_stats(self, _c.byref(st)), "ridfa_server_get_stats")
        return st.as_dict()

    def close(self):
        if self.handle:
            _lib.ridfa_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        if not self.handle:
            raise ValueError("server is closed")
        return self.handle


# ------------------------------------------------------------------------------ diagnostics
class TransitionCounts(_c.Structure):
    _fields_ = [("w_paper", _c.c_uint64), ("w_conv", _c.c_uint64), ("runs", _c.c_uint64),
                ("dead_runs", _c.c_uint64), ("converge_hist", _c.c_uint64 * 16)]


_decl("ridfa_count_transitions", _c.c_int, [_vp, _c.c_int, _vp, _c.c_size_t, _u32, _u32,
                                            _c.POINTER(TransitionCounts)])


def ridfa_count_transitions(prog, text, n_chunks, dfa=False, n_threads=0, nfa=False):
    """Host transition counts of the reach phase over a host text (bytes or uint8 array):
    dict with w_paper, w_conv, runs, dead_runs and converge_hist (16 log2 buckets of the bytes
    until a chunk's runs leave one live state; the last: never); dfa=True for the all-states DFA
    comparator, nfa=True for the NFA variant."""
    if isinstance(text, (bytes, bytearray)):
        buf = np.frombuffer(text, dtype=np.uint8)
    else:
        buf = np.ascontiguousarray(text, dtype=np.uint8)
    out = TransitionCounts()
    which = 2 if nfa else int(bool(dfa))
    _check(_lib.ridfa_count_transitions(prog, which, buf.ctypes.data if buf.size else None, buf.size,
                                        int(n_chunks), int(n_threads), _c.byref(out)), "ridfa_count_transitions")
    return {f: (list(getattr(out, f)) if f == "converge_hist" else getattr(out, f)) for f, _ in out._fields_}


_decl("ridfa_cpu_recognize", _c.c_int, [_vp, _c.c_int, _vp, _c.c_size_t, _u32, _u32, _c.POINTER(_c.c_uint8)])


def ridfa_cpu_recognize(prog, text, n_chunks, dfa=False, n_threads=0):
    """The recognition on the host's cores (a comparison, never a fallback): n_chunks = 1 is
    the serial table loop, n_chunks > 1 the chunked speculative run on n_threads threads (0 =
    all); dfa=True for the all-states DFA variant.  Returns the accept bit."""
    if isinstance(text, (bytes, bytearray)):
        buf = np.frombuffer(text, dtype=np.uint8)
    else:
        buf = np.ascontiguousarray(text, dtype=np.uint8)
    acc = _c.c_uint8(0)
    _check(_lib.ridfa_cpu_recognize(prog, int(bool(dfa)), buf.ctypes.data if buf.size else None, buf.size,
                                    int(n_chunks), int(n_threads), _c.byref(acc)), "ridfa_cpu_recognize")
    return bool(acc.value)


# ---------------------------------------------------------------------------------- shards
class ShardSummary(_c.Structure):
    _fields_ = [("k", _u32), ("n_out", _u32), ("entry", _c.c_uint16 * RIDFA_MAX_SLOTS),
                ("out_state", _c.c_uint16 * RIDFA_MAX_SLOTS),
                ("reach", (_u32 * (RIDFA_MAX_SLOTS // 32)) * RIDFA_MAX_SLOTS)]

    def to_bytes(self):
        return bytes(self)

    @classmethod
    def from_bytes(cls, b):
        return cls.from_buffer_copy(bytes(b))


_decl("ridfa_recognize_shard", _c.c_int, [_vp, _vp, _c.c_size_t, _u32, _c.POINTER(Tuning),
                                          _c.POINTER(ShardSummary), _vp])
_decl("ridfa_join_shards", _c.c_int, [_vp, _c.POINTER(ShardSummary), _u32, _c.POINTER(_c.c_uint8)])


def ridfa_recognize_shard(prog, d_text, length, n_chunks, tuning=None, stream=None):
    """Relation summary of one shard of a text (device pointer / tensor), as a ShardSummary."""
    out = ShardSummary()
    _check(_lib.ridfa_recognize_shard(prog, _ptr(d_text), int(length), int(n_chunks), _tuning(tuning),
                                      _c.byref(out), _stream(stream)), "ridfa_recognize_shard")
    return out


def ridfa_join_shards(prog, summaries):
    """Accept bit of the text made of consecutive shards, from their summaries (host only)."""
    arr = (ShardSummary * len(summaries))(*summaries)
    acc = _c.c_uint8(0)
    _check(_lib.ridfa_join_shards(prog, arr, len(summaries), _c.byref(acc)), "ridfa_join_shards")
    return bool(acc.value)


# ------------------------------------------------------------------------------ join scan
_decl("ridfa_join_scan", _c.c_int, [_vp, _vp, _u32, _vp, _c.POINTER(_c.c_int64), _vp])


def ridfa_join_scan(prog, d_maps, n_chunks, d_entry=None, stream=None):
    """Per-chunk entry sets E_i into d_entry (device uint32 [n_chunks][ceil(k/32)], optional);
    returns the first rejecting chunk or -1."""
    rej = _c.c_int64(0)
    _check(_lib.ridfa_join_scan(prog, _ptr(d_maps), int(n_chunks), _ptr(d_entry), _c.byref(rej), _stream(stream)),
           "ridfa_join_scan")
    return rej.value
