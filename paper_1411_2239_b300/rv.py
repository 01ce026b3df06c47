"""Thin ctypes binding of librv (include/rv.h): argument marshalling only.

Every step of verification runs inside librv's CUDA kernels; this module only
converts Python/NumPy/PyTorch arguments into the C structs and back.  PyTorch
provides device memory (workspaces, outputs) and streams.  The library must
be built (``python -m paper_1411_2239_b300.build``); loading fails loudly
otherwise -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librv.so")

RV_OK, RV_EPARSE, RV_EUNSUPPORTED, RV_EINVAL, RV_ENOMEM, RV_EAGAIN, RV_ETIMEOUT, RV_ECUDA, RV_EINTERNAL = range(9)
STATUS_NAMES = ["RV_OK", "RV_EPARSE", "RV_EUNSUPPORTED", "RV_EINVAL", "RV_ENOMEM", "RV_EAGAIN",
                "RV_ETIMEOUT", "RV_ECUDA", "RV_EINTERNAL"]
ONEHOT, BITMASK = 0, 1
Q_A, Q_E = 0, 1
OPS = {"<": 0, "<=": 1, ">": 2, ">=": 3, "=": 4}
VERDICT_NAMES = ["F", "Fc", "Fp", "Tp", "Tc", "T"]


class RVError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class _Schema(ctypes.Structure):
    _fields_ = [("n_codes", ctypes.c_int), ("code_names", ctypes.POINTER(ctypes.c_char_p)),
                ("alphabet", ctypes.c_int), ("key_bits", ctypes.c_int), ("value_name", ctypes.c_char_p)]


class _Info(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in ("n_quant", "n_states", "n_letters", "q0", "key_bits", "alphabet",
                                            "n_base", "n_cmp")]


class _Trace(ctypes.Structure):
    _fields_ = [("key", ctypes.c_void_p), ("pred", ctypes.c_void_p), ("ts", ctypes.c_void_p), ("n", ctypes.c_uint64),
                ("value", ctypes.c_void_p)]


class _Result(ctypes.Structure):
    _fields_ = [("root", ctypes.c_int32), ("status", ctypes.c_int32), ("root_counts", ctypes.c_uint64 * 6),
                ("level_counts", (ctypes.c_uint64 * 6) * 2), ("n_nodes", ctypes.c_uint64 * 2),
                ("events", ctypes.c_uint64)]


class _Bindings(ctypes.Structure):
    _fields_ = [("keys", ctypes.c_void_p), ("verdicts", ctypes.c_void_p), ("capacity", ctypes.c_uint64),
                ("outer_keys", ctypes.c_void_p), ("outer_verdicts", ctypes.c_void_p),
                ("outer_capacity", ctypes.c_uint64)]


class _Opts(ctypes.Structure):
    _fields_ = [("bucket_bits", ctypes.c_int), ("sub_bucket_bits", ctypes.c_int), ("unit_records", ctypes.c_int),
                ("no_heavy", ctypes.c_int), ("test_wait_polls", ctypes.c_int)]


RESULT_BYTES = ctypes.sizeof(_Result)
_lib = None


def lib():
    """Load librv.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"librv.so not built at {LIB_PATH}; run python -m paper_1411_2239_b300.build")
        L = ctypes.CDLL(LIB_PATH)
        vp, u64, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
        L.rv_compile_formula.argtypes = [ctypes.c_char_p, ctypes.POINTER(_Schema), ctypes.POINTER(vp),
                                         ctypes.c_char_p, ctypes.c_size_t]
        L.rv_formula_get_info.argtypes = [vp, ctypes.POINTER(_Info)]
        L.rv_formula_tables.argtypes = [vp, ctypes.POINTER(u64), i32, ctypes.POINTER(ctypes.c_uint8)]
        L.rv_formula_quantifier.argtypes = [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                            ctypes.POINTER(u64), ctypes.POINTER(u64)]
        L.rv_formula_free.argtypes = [vp]
        L.rv_formula_free.restype = None
        L.rv_valuate.argtypes = [i32, i32, u64, u64, ctypes.POINTER(u64), ctypes.POINTER(i32)]
        L.rv_verify_workspace_size.argtypes = [vp, u64, i32, ctypes.POINTER(_Opts)]
        L.rv_verify_workspace_size.restype = ctypes.c_size_t
        L.rv_verify_trace.argtypes = [vp, ctypes.POINTER(_Trace), i32, vp, ctypes.c_size_t, ctypes.POINTER(_Result),
                                      ctypes.POINTER(_Bindings), ctypes.POINTER(_Opts), vp]
        L.rv_verify_trace_async.argtypes = [vp, ctypes.POINTER(_Trace), vp, ctypes.c_size_t, vp,
                                            ctypes.POINTER(_Bindings), ctypes.POINTER(_Opts), vp]
        L.rv_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def last_error() -> str:
    return lib().rv_last_error().decode()


def _check(st):
    if st != RV_OK:
        raise RVError(st, last_error())


@dataclass
class Quantifier:
    kind: int
    op: int
    num: int
    den: int


class Formula:
    """A compiled LTL4-C formula (owns an rv_formula)."""

    def __init__(self, text: str, codes, alphabet: str = "onehot", key_bits: int = 32, value_name=None):
        L = lib()
        self.text, self.codes = text, list(codes)
        self.alphabet = ONEHOT if alphabet == "onehot" else BITMASK
        names = (ctypes.c_char_p * len(self.codes))(*[c.encode() for c in self.codes])
        self._names = names
        self._value_name = None if value_name is None else value_name.encode()
        sch = _Schema(len(self.codes), names, self.alphabet, key_bits, self._value_name)
        h = ctypes.c_void_p()
        err = ctypes.create_string_buffer(512)
        st = L.rv_compile_formula(text.encode(), ctypes.byref(sch), ctypes.byref(h), err, 512)
        if st != RV_OK:
            raise RVError(st, err.value.decode())
        self._h = h
        info = _Info()
        _check(L.rv_formula_get_info(h, ctypes.byref(info)))
        self.n_quant, self.n_states, self.n_letters = info.n_quant, info.n_states, info.n_letters
        self.q0, self.key_bits = info.q0, info.key_bits
        self.n_base, self.n_cmp = info.n_base, info.n_cmp

    @property
    def handle(self):
        return self._h

    def tables(self):
        maps = (ctypes.c_uint64 * self.n_letters)()
        labels = (ctypes.c_uint8 * 16)()
        _check(lib().rv_formula_tables(self._h, maps, self.n_letters, labels))
        return [int(m) for m in maps], [int(x) for x in labels]

    def quantifier(self, level):
        k, o = ctypes.c_int(), ctypes.c_int()
        n, d = ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib().rv_formula_quantifier(self._h, level, ctypes.byref(k), ctypes.byref(o), ctypes.byref(n),
                                           ctypes.byref(d)))
        return Quantifier(k.value, o.value, n.value, d.value)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.rv_formula_free(h)
            self._h = None


def valuate(kind, op, num, den, v) -> int:
    arr = (ctypes.c_uint64 * 6)(*[int(x) for x in v])
    out = ctypes.c_int()
    _check(lib().rv_valuate(kind, op, num, den, arr, ctypes.byref(out)))
    return out.value


@dataclass
class Result:
    root: int
    status: int
    root_counts: list
    level_counts: list
    n_nodes: list
    events: int
    bindings: dict = field(default_factory=dict)
    outer: dict = field(default_factory=dict)


def _result(r: _Result) -> Result:
    return Result(r.root, r.status, list(r.root_counts), [list(r.level_counts[0]), list(r.level_counts[1])],
                  list(r.n_nodes), r.events)


def _opts(opts):
    if not opts:
        return None
    return ctypes.byref(_Opts(opts.get("bucket_bits", 0), opts.get("sub_bucket_bits", 0), opts.get("unit_records", 0),
                              int(opts.get("no_heavy", 0)), int(opts.get("test_wait_polls", 0))))


def workspace_size(formula: Formula, n: int, host_input: bool = False, opts=None) -> int:
    return int(lib().rv_verify_workspace_size(formula.handle, n, int(host_input), _opts(opts)))


_ws_cache = {}


def workspace(nbytes: int, device=None):
    """A cached torch uint8 buffer of at least nbytes on the current device."""
    import torch
    if device is None:
        device = torch.device("cuda", torch.cuda.current_device())
    buf = _ws_cache.get(device)
    if buf is None or buf.numel() < nbytes:
        _ws_cache.pop(device, None)
        buf = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=device)
        _ws_cache[device] = buf
    return buf


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def verify(formula: Formula, key, pred, ts=None, stream=None, want_bindings=False, opts=None, ws=None,
           value=None) -> Result:
    """Verify one trace.  key/pred/ts/value: torch CUDA tensors (device path)
    or NumPy arrays (host path: copied in by the library)."""
    import torch
    on_device = isinstance(pred, torch.Tensor) and pred.is_cuda
    if not on_device:
        key = np.ascontiguousarray(key)
        pred = np.ascontiguousarray(pred, dtype=np.uint8)
        ts = None if ts is None else np.ascontiguousarray(ts, dtype=np.uint32)
        value = None if value is None else np.ascontiguousarray(value, dtype=np.uint32)
        want_kb = 8 if formula.key_bits == 64 else 4
        if key.dtype.itemsize != want_kb:
            key = key.astype(np.uint64 if want_kb == 8 else np.uint32)
    n = int(pred.shape[0])
    tr = _Trace(_ptr(key), _ptr(pred), _ptr(ts), n, _ptr(value))
    need = workspace_size(formula, n, not on_device, opts)
    if ws is None:
        ws = workspace(need)
    binds = None
    outs = {}
    if want_bindings:
        cap = max(n, 1)
        outs = {"keys": torch.empty(cap, dtype=torch.int64, device="cuda"),
                "verdicts": torch.empty(cap, dtype=torch.uint8, device="cuda"),
                "okeys": torch.empty(cap, dtype=torch.int64, device="cuda"),
                "overdicts": torch.empty(cap, dtype=torch.uint8, device="cuda")}
        binds = ctypes.byref(_Bindings(outs["keys"].data_ptr(), outs["verdicts"].data_ptr(), cap,
                                       outs["okeys"].data_ptr(), outs["overdicts"].data_ptr(), cap))
    r = _Result()
    _check(lib().rv_verify_trace(formula.handle, ctypes.byref(tr), int(on_device), ctypes.c_void_p(ws.data_ptr()),
                                 ws.numel(), ctypes.byref(r), binds, _opts(opts), _stream_handle(stream)))
    res = _result(r)
    if want_bindings:
        if formula.n_quant == 2:
            ni, no = int(res.n_nodes[1]), int(res.n_nodes[0])
        else:
            ni, no = int(res.n_nodes[0]), 0
        k = outs["keys"][:ni].cpu().numpy().view(np.uint64)
        v = outs["verdicts"][:ni].cpu().numpy()
        res.bindings = dict(zip(k.tolist(), v.tolist()))
        if no:
            k = outs["okeys"][:no].cpu().numpy().view(np.uint64)
            v = outs["overdicts"][:no].cpu().numpy()
            res.outer = dict(zip(k.tolist(), v.tolist()))
    return res


def verify_async(formula: Formula, key, pred, ws, dev_result, stream=None, opts=None, ts=None, value=None):
    """Enqueue verification of a device-resident trace; the result lands in
    dev_result (a torch uint8 CUDA tensor of RESULT_BYTES bytes)."""
    n = int(pred.shape[0])
    tr = _Trace(_ptr(key), _ptr(pred), _ptr(ts), n, _ptr(value))
    _check(lib().rv_verify_trace_async(formula.handle, ctypes.byref(tr), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                       ctypes.c_void_p(dev_result.data_ptr()), None, _opts(opts),
                                       _stream_handle(stream)))


def parse_result(raw: bytes) -> Result:
    r = _Result.from_buffer_copy(raw)
    return _result(r)


# ---------------------------------------------------------------------- front end: strace text
KEY_ARG0, KEY_RET = 0, 1


class _Rule(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("code", ctypes.c_int), ("key_from", ctypes.c_int),
                ("ok_only", ctypes.c_int)]


def parse_strace(text, rules, capacity=None, stream=None):
    """Event table of a strace log (rv_parse_strace).  text: bytes/str (copied
    to the device) or a torch uint8 CUDA tensor; rules: (name, code, key_from,
    ok_only) tuples.  Returns device tensors (key int32 view of uint32, pred
    uint8, ts int64 microseconds) of the events."""
    import torch
    L = lib()
    if not getattr(L, "_parse_sigs", False):
        vp = ctypes.c_void_p
        L.rv_parse_workspace_size.argtypes = [ctypes.c_uint64]
        L.rv_parse_workspace_size.restype = ctypes.c_size_t
        L.rv_parse_strace.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(_Rule), ctypes.c_int, vp, ctypes.c_size_t,
                                      vp, vp, vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64), vp]
        L._parse_sigs = True
    if isinstance(text, str):
        text = text.encode()
    if not isinstance(text, torch.Tensor):
        text = torch.frombuffer(bytearray(text), dtype=torch.uint8).cuda() if len(text) else \
            torch.empty(0, dtype=torch.uint8, device="cuda")
    nbytes = int(text.numel())
    cap = capacity if capacity is not None else max(1, nbytes // 16 + 1)
    names = [r[0].encode() for r in rules]
    arr = (_Rule * len(rules))(*[_Rule(nm, int(r[1]), int(r[2]), int(r[3]) if len(r) > 3 else 0)
                                 for nm, r in zip(names, rules)])
    key = torch.empty(cap, dtype=torch.int32, device=text.device)
    pred = torch.empty(cap, dtype=torch.uint8, device=text.device)
    ts = torch.empty(cap, dtype=torch.int64, device=text.device)
    ws = workspace(int(L.rv_parse_workspace_size(nbytes)))
    n = ctypes.c_uint64()
    _check(L.rv_parse_strace(_ptr(text) if nbytes else None, nbytes, arr, len(rules), ctypes.c_void_p(ws.data_ptr()),
                             ws.numel(), _ptr(key), _ptr(pred), _ptr(ts), cap, ctypes.byref(n),
                             _stream_handle(stream)))
    k = n.value
    return key[:k], pred[:k], ts[:k]


# ---------------------------------------------------------------------- per-event timeline
def timeline(formula: Formula, key, pred, stream=None, value=None):
    """Per-event verdicts and first violations of a device trace
    (rv_verify_timeline).  Returns (verdicts: np.uint8[n] in trace order,
    first_violation: {binding key: event index})."""
    verd, vkey, vidx, k = timeline_device(formula, key, pred, stream, value)
    keys = vkey[:k].cpu().numpy().view(np.uint64).tolist()
    idx = vidx[:k].cpu().numpy().view(np.uint32).tolist()
    return verd.cpu().numpy(), dict(zip(keys, idx))


def timeline_device(formula: Formula, key, pred, stream=None, value=None, out=None):
    """rv_verify_timeline into device tensors: (verdicts uint8[n], violation
    keys, violation indices, number of violations).  `out` reuses the output
    tensors of an earlier call of the same size."""
    import torch
    L = lib()
    if not getattr(L, "_tl_sigs", False):
        vp = ctypes.c_void_p
        L.rv_timeline_workspace_size.argtypes = [vp, ctypes.c_uint64]
        L.rv_timeline_workspace_size.restype = ctypes.c_size_t
        L.rv_verify_timeline.argtypes = [vp, ctypes.POINTER(_Trace), vp, ctypes.c_size_t, vp, vp, vp, vp, vp]
        L._tl_sigs = True
    n = int(pred.shape[0])
    dev = pred.device
    if out is None:
        out = (torch.empty(max(n, 1), dtype=torch.uint8, device=dev), torch.empty(max(n, 1), dtype=torch.int64, device=dev),
               torch.empty(max(n, 1), dtype=torch.int32, device=dev), torch.zeros(1, dtype=torch.int64, device=dev))
    verd, vkey, vidx, nv = out
    ws = workspace(int(L.rv_timeline_workspace_size(formula.handle, n)))
    tr = _Trace(_ptr(key), _ptr(pred), None, n, _ptr(value))
    _check(L.rv_verify_timeline(formula.handle, ctypes.byref(tr), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                _ptr(verd), _ptr(vkey), _ptr(vidx), _ptr(nv), _stream_handle(stream)))
    timeline_device.last_out = out
    return verd[:n], vkey, vidx, int(nv.item())


# ---------------------------------------------------------------------- one trace over several ranks
def _shard_sigs(L):
    if getattr(L, "_shard_sigs", False):
        return
    vp, u64 = ctypes.c_void_p, ctypes.c_uint64
    L.rv_shard_of.argtypes = [vp, vp, u64, ctypes.c_int, vp]
    L.rv_shard_workspace_size.argtypes = [u64, ctypes.c_int]
    L.rv_shard_workspace_size.restype = ctypes.c_size_t
    L.rv_shard_trace.argtypes = [vp, ctypes.POINTER(_Trace), ctypes.c_int, vp, ctypes.c_size_t, vp, vp, vp, vp, vp,
                                 vp]
    L.rv_combine_results.argtypes = [vp, ctypes.POINTER(_Result), ctypes.c_int, ctypes.POINTER(_Result)]
    L._shard_sigs = True


def shard_of(formula: Formula, key, world: int) -> np.ndarray:
    """Rank in [0, world) of every event of a host key array (rv_shard_of)."""
    L = lib()
    _shard_sigs(L)
    key = np.ascontiguousarray(key, dtype=np.uint64 if formula.key_bits == 64 else np.uint32)
    out = np.empty(len(key), dtype=np.uint32)
    _check(L.rv_shard_of(formula.handle, key.ctypes.data, len(key), world, out.ctypes.data))
    return out


def shard_trace(formula: Formula, key, pred, world: int, ts=None, stream=None, value=None):
    """Group a device trace into world contiguous segments by rank (rv_shard_trace).
    Returns (key_out, pred_out, ts_out or None, counts) with counts a device
    uint64 tensor (as int64) of the segment sizes; with value, the moved
    values are in the attribute shard_trace.last_value."""
    import torch
    L = lib()
    _shard_sigs(L)
    n = int(pred.shape[0])
    key_out = torch.empty_like(key)
    pred_out = torch.empty_like(pred)
    ts_out = None if ts is None else torch.empty_like(ts)
    value_out = None if value is None else torch.empty_like(value)
    counts = torch.empty(world, dtype=torch.int64, device=pred.device)
    ws = workspace(int(L.rv_shard_workspace_size(n, world)))
    tr = _Trace(_ptr(key), _ptr(pred), _ptr(ts), n, _ptr(value))
    _check(L.rv_shard_trace(formula.handle, ctypes.byref(tr), world, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                            _ptr(key_out), _ptr(pred_out), _ptr(ts_out), _ptr(value_out), _ptr(counts),
                            _stream_handle(stream)))
    shard_trace.last_value = value_out
    return key_out, pred_out, ts_out, counts


def _to_c(r: Result) -> _Result:
    c = _Result()
    c.root, c.status, c.events = r.root, r.status, r.events
    for v in range(6):
        c.root_counts[v] = r.root_counts[v]
        c.level_counts[0][v] = r.level_counts[0][v]
        c.level_counts[1][v] = r.level_counts[1][v]
    c.n_nodes[0], c.n_nodes[1] = r.n_nodes
    return c


def combine_results(formula: Formula, parts) -> Result:
    """The whole trace's result from its parts' results (rv_combine_results)."""
    L = lib()
    _shard_sigs(L)
    arr = (_Result * len(parts))(*[_to_c(p) for p in parts])
    out = _Result()
    _check(L.rv_combine_results(formula.handle, arr, len(parts), ctypes.byref(out)))
    return _result(out)


# ---------------------------------------------------------------------- batched
class _BatchOpts(ctypes.Structure):
    _fields_ = [("bucket_records", ctypes.c_int), ("tile_events", ctypes.c_int), ("long_records", ctypes.c_int)]


def _batch_sigs(L):
    if getattr(L, "_batch_sigs", False):
        return
    vp = ctypes.c_void_p
    L.rv_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64),
                                  ctypes.POINTER(_BatchOpts), ctypes.POINTER(vp)]
    L.rv_batch_workspace_size.argtypes = [vp]
    L.rv_batch_workspace_size.restype = ctypes.c_size_t
    L.rv_batch_run.argtypes = [vp, vp, vp, vp, ctypes.c_size_t, vp, vp]
    L.rv_batch_autotune.argtypes = [vp, vp, vp, vp, ctypes.c_size_t, vp, vp, ctypes.POINTER(_BatchOpts)]
    L.rv_batch_free.argtypes = [vp]
    L.rv_batch_free.restype = None
    L._batch_sigs = True


class Batch:
    """Many traces (concatenated, CSR offsets) x nf formulas per trace, run as
    one captured graph (rv_batch_*)."""

    def __init__(self, formulas, offsets, bucket_records=0, tile_events=0, long_records=0):
        L = lib()
        _batch_sigs(L)
        self.nt = len(formulas)
        self.nf = len(formulas[0])
        self._keep = formulas
        flat = (ctypes.c_void_p * (self.nt * self.nf))(*[f.handle.value for fs in formulas for f in fs])
        self.offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        h = ctypes.c_void_p()
        opts = _BatchOpts(bucket_records, tile_events, long_records)
        _check(L.rv_batch_create(flat, self.nf, self.nt, self.offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                 ctypes.byref(opts), ctypes.byref(h)))
        self._h = h

    def workspace_size(self):
        return int(lib().rv_batch_workspace_size(self._h))

    def run(self, key, pred, ws, dev_results, stream=None):
        _check(lib().rv_batch_run(self._h, ctypes.c_void_p(key.data_ptr()), ctypes.c_void_p(pred.data_ptr()),
                                  ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.c_void_p(dev_results.data_ptr()),
                                  _stream_handle(stream)))

    def autotune(self, key, pred, ws, dev_results, stream=None):
        ch = _BatchOpts()
        _check(lib().rv_batch_autotune(self._h, ctypes.c_void_p(key.data_ptr()), ctypes.c_void_p(pred.data_ptr()),
                                       ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                       ctypes.c_void_p(dev_results.data_ptr()), _stream_handle(stream),
                                       ctypes.byref(ch)))
        return {"bucket_records": ch.bucket_records, "tile_events": ch.tile_events, "long_records": ch.long_records}

    def results(self, dev_results):
        raw = bytes(dev_results.cpu().numpy())
        return [_result(_Result.from_buffer_copy(raw, i * RESULT_BYTES)) for i in range(self.nt * self.nf)]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.rv_batch_free(h)
            self._h = None


# ---------------------------------------------------------------------- serving
class _SvcCfg(ctypes.Structure):
    _fields_ = [("max_bindings", ctypes.c_uint64), ("max_outer", ctypes.c_uint64),
                ("max_batch_events", ctypes.c_uint64), ("max_staged_events", ctypes.c_uint64),
                ("max_streams", ctypes.c_int)]


class _Verdict(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("root", ctypes.c_int32), ("status", ctypes.c_int32),
                ("root_counts", ctypes.c_uint64 * 6), ("events", ctypes.c_uint64), ("latency_us", ctypes.c_double)]


class _SvcCounters(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("batches", "admitted", "refused", "events", "bindings",
                                              "outer_nodes", "staged_events")]


def _svc_sigs(L):
    if getattr(L, "_svc_sigs", False):
        return
    vp = ctypes.c_void_p
    L.rv_service_open.argtypes = [vp, ctypes.POINTER(_SvcCfg), ctypes.POINTER(vp)]
    L.rv_service_close.argtypes = [vp]
    L.rv_stream_open.argtypes = [vp, ctypes.POINTER(vp)]
    L.rv_stream_push.argtypes = [vp, ctypes.POINTER(_Trace), ctypes.POINTER(ctypes.c_uint64)]
    L.rv_stream_poll.argtypes = [vp, ctypes.POINTER(_Verdict), ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int]
    L.rv_stream_close.argtypes = [vp]
    L.rv_service_stats.argtypes = [vp, ctypes.POINTER(_SvcCounters)]
    L._svc_sigs = True


@dataclass
class StreamVerdict:
    ticket: int
    root: int
    status: int
    root_counts: list
    events: int
    latency_us: float


class Service:
    """Online verification service (rv_service_*): continuous batching of chunks
    from many streams, monitor state resident on the GPU."""

    def __init__(self, formula: Formula, max_bindings=0, max_outer=0, max_batch_events=0, max_staged_events=0,
                 max_streams=0):
        L = lib()
        _svc_sigs(L)
        self.formula = formula
        cfg = _SvcCfg(max_bindings, max_outer, max_batch_events, max_staged_events, max_streams)
        h = ctypes.c_void_p()
        _check(L.rv_service_open(formula.handle, ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h

    def open_stream(self):
        h = ctypes.c_void_p()
        _check(lib().rv_stream_open(self._h, ctypes.byref(h)))
        return Stream(self, h)

    def stats(self):
        c = _SvcCounters()
        _check(lib().rv_service_stats(self._h, ctypes.byref(c)))
        return {n: getattr(c, n) for n, _ in _SvcCounters._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().rv_service_close(self._h)
            self._h = None

    def __del__(self):
        self.close()


class Stream:
    """A stream of a Service.  close() ends it: the library frees the handle
    once its queued work is retired, so a closed Stream refuses further calls."""

    def __init__(self, svc, h):
        self.svc, self._h = svc, h

    def _handle(self):
        if self._h is None:
            raise RVError(RV_EINVAL, "stream is closed")
        return self._h

    def push(self, key, pred, ts=None):
        """Stage a chunk (host arrays); returns its ticket; raises RVError(RV_EAGAIN) if not admitted."""
        h = self._handle()
        key = np.ascontiguousarray(key)
        pred = np.ascontiguousarray(pred, dtype=np.uint8)
        tr = _Trace(key.ctypes.data, pred.ctypes.data, None if ts is None else np.ascontiguousarray(ts).ctypes.data,
                    len(pred))
        t = ctypes.c_uint64()
        st = lib().rv_stream_push(h, ctypes.byref(tr), ctypes.byref(t))
        if st != RV_OK:
            raise RVError(st, last_error())
        return t.value

    def poll(self, max_n=64, timeout_us=0):
        buf = (_Verdict * max_n)()
        n = ctypes.c_int()
        st = lib().rv_stream_poll(self._handle(), buf, max_n, ctypes.byref(n), int(timeout_us))
        if st == RV_ETIMEOUT:
            return []
        if st != RV_OK:
            raise RVError(st, last_error())
        return [StreamVerdict(v.ticket, v.root, v.status, list(v.root_counts), v.events, v.latency_us)
                for v in buf[:n.value]]

    def close(self):
        if self._h is not None:
            lib().rv_stream_close(self._h)
            self._h = None
