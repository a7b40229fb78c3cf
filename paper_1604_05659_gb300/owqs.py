"""Python binding of libowqs.so (ctypes; argument marshalling only).

Every step of a simulation runs in the library's CUDA kernels; this module
only converts patterns, options and buffers into the C ABI of include/owqs.h.
If the library has not been built, library() raises: there is no Python or
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libowqs.so")

OK, ERR_ARG, ERR_PATTERN, ERR_NOT_STANDARD, ERR_IMPOSSIBLE_BRANCH, ERR_NOT_DETERMINISTIC, \
    ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED = range(10)
STATUS_NAMES = ["OK", "ERR_ARG", "ERR_PATTERN", "ERR_NOT_STANDARD", "ERR_IMPOSSIBLE_BRANCH",
                "ERR_NOT_DETERMINISTIC", "ERR_OOM", "ERR_CUDA", "ERR_TIMEOUT", "ERR_UNSUPPORTED"]
CMD_KIND = {"N": 0, "E": 1, "M": 2, "X": 3, "Z": 4}
MODE = {"owqs": 0, "eowqs": 1}
FLOW_CAUSAL, FLOW_GFLOW = 0, 1
RUN_HOST_SAMPLING = 1
RUN_PER_PASS = 2
RUN_SEQUENTIAL_SAMPLING = 4
RUN_SUBSTATES = 8
RUN_ONE_ARRAY = 16
RUN_DOUBLE_FLOAT = 32
DTYPE = {"c64": 0, "c128": 1}
POLICY = {"forced": 0, "sampled": 1, "zero": 2}
KERNEL_KIND = {0: "fast_pass", 1: "generic_pass", 2: "final", 3: "norm", 4: "prob", 5: "tma_pass", 10: "small_run",
               7: "decide", 8: "group_pass", 9: "factor_join", 11: "tma_prob"}


class OwqsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class owqs_cmd(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("q0", C.c_uint32), ("q1", C.c_uint32), ("pad_", C.c_uint32),
                ("angle", C.c_double), ("s_off", C.c_uint32), ("s_len", C.c_uint32),
                ("t_off", C.c_uint32), ("t_len", C.c_uint32)]


class owqs_pattern_info(C.Structure):
    _fields_ = [("nqubits", C.c_uint32), ("nin", C.c_uint32), ("nout", C.c_uint32), ("nmeas", C.c_uint32),
                ("standard", C.c_uint32), ("peak_live", C.c_uint32), ("amp_updates", C.c_uint64)]


class owqs_reorder_opts(C.Structure):
    _fields_ = [("mode", C.c_uint32), ("product_input", C.c_uint32), ("sweep", C.c_uint32),
                ("use_learned", C.c_uint32), ("alpha", C.c_double), ("beta", C.c_double),
                ("gamma", C.c_double), ("delta", C.c_double), ("model", C.c_void_p)]


class owqs_reorder_info(C.Structure):
    _fields_ = [("peak_m", C.c_uint32), ("peak_live", C.c_uint32), ("amp_updates", C.c_uint64),
                ("alpha_used", C.c_double), ("learned_accepted", C.c_uint32), ("greedy_peak_live", C.c_uint32),
                ("greedy_amp_updates", C.c_uint64), ("learned_peak_live", C.c_uint32),
                ("greedy_best_owqs", C.c_uint32), ("learned_amp_updates", C.c_uint64)]


class owqs_run_opts(C.Structure):
    _fields_ = [("dtype", C.c_uint32), ("mode", C.c_uint32), ("policy", C.c_uint32), ("io", C.c_uint32),
                ("seed", C.c_uint64), ("stream", C.c_void_p), ("use_graph", C.c_uint32), ("flags", C.c_uint32)]


class owqs_memory_plan(C.Structure):
    _fields_ = [("peak_m", C.c_uint32), ("components", C.c_uint32), ("joins", C.c_uint32),
                ("uses_substates", C.c_uint32), ("substate_bytes", C.c_uint64), ("one_array_bytes", C.c_uint64),
                ("substate_work", C.c_double), ("one_array_work", C.c_double)]


class owqs_sample_info(C.Structure):
    _fields_ = [("path", C.c_uint32), ("guessed", C.c_uint32), ("checks", C.c_uint32), ("relaunches", C.c_uint32)]


SAMPLE_PATH = {0: "none", 1: "drawn_first", 2: "guess_kept", 3: "checked_launches", 4: "one_at_a_time",
               5: "host"}


class owqs_batch_item(C.Structure):
    _fields_ = [("pattern", C.c_void_p), ("outcomes", C.POINTER(C.c_uint8)), ("psi_in", C.c_void_p),
                ("out", C.c_void_p), ("ref", C.c_int32), ("pad_", C.c_uint32)]


_BATCH_ITEM_DTYPE = np.dtype([("pattern", np.uint64), ("outcomes", np.uint64), ("psi_in", np.uint64),
                              ("out", np.uint64), ("ref", np.int32), ("pad_", np.uint32)])
assert _BATCH_ITEM_DTYPE.itemsize == C.sizeof(owqs_batch_item)


class owqs_batch_opts(C.Structure):
    _fields_ = [("dtype", C.c_uint32), ("column_block", C.c_uint32), ("stream", C.c_void_p),
                ("use_graph", C.c_uint32), ("pad_", C.c_uint32), ("overlaps", C.POINTER(C.c_double))]


class owqs_batch_info(C.Structure):
    _fields_ = [("smem_items", C.c_uint32), ("hbm_items", C.c_uint32), ("tasks", C.c_uint32),
                ("smem_bytes_per_cta", C.c_uint32), ("launches", C.c_uint32), ("global_items", C.c_uint32),
                ("compile_ms", C.c_float), ("call_ms", C.c_float)]


class owqs_pass_desc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_in", C.c_int32), ("r", C.c_int32), ("b", C.c_int32),
                ("n_out", C.c_int32), ("outcome", C.c_int32), ("xmask", C.c_uint64), ("zmask", C.c_uint64),
                ("c0", C.c_uint32), ("nedges", C.c_uint32), ("edges", (C.c_uint32 * 2) * 64),
                ("w1re", C.c_double), ("w1im", C.c_double), ("scale", C.c_double), ("perm", C.c_int32 * 64)]


EXPORTS = {
    "owqs_load_pattern": (C.c_int, [C.c_uint32, C.POINTER(C.c_uint32), C.c_uint32, C.POINTER(C.c_uint32),
                                    C.c_uint32, C.POINTER(owqs_cmd), C.c_size_t, C.POINTER(C.c_uint32),
                                    C.c_size_t, C.POINTER(C.c_void_p)]),
    "owqs_free_pattern": (None, [C.c_void_p]),
    "owqs_get_info": (C.c_int, [C.c_void_p, C.POINTER(owqs_pattern_info)]),
    "owqs_reorder": (C.c_int, [C.c_void_p, C.POINTER(owqs_reorder_opts), C.POINTER(owqs_reorder_info),
                               C.POINTER(C.c_uint32)]),
    "owqs_set_order": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint32), C.c_uint32]),
    "owqs_reset_order": (C.c_int, [C.c_void_p]),
    "owqs_get_order": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint32)]),
    "owqs_run": (C.c_int, [C.c_void_p, C.POINTER(owqs_run_opts), C.c_void_p, C.c_void_p,
                           C.POINTER(C.c_uint8), C.POINTER(C.c_double)]),
    "owqs_run_async": (C.c_int, [C.c_void_p, C.POINTER(owqs_run_opts), C.c_void_p, C.c_void_p,
                                 C.POINTER(C.c_uint8)]),
    "owqs_wait": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint8), C.POINTER(C.c_double)]),
    "owqs_unitary": (C.c_int, [C.c_void_p, C.POINTER(owqs_run_opts), C.POINTER(C.c_uint8), C.c_void_p,
                               C.POINTER(C.c_double)]),
    "owqs_run_batch": (C.c_int, [C.POINTER(owqs_batch_item), C.c_uint32, C.POINTER(owqs_batch_opts),
                                 C.POINTER(owqs_batch_info)]),
    "owqs_run_static": (C.c_int, [C.c_void_p, C.POINTER(owqs_run_opts), C.c_void_p, C.c_void_p,
                                  C.POINTER(C.c_uint8), C.POINTER(C.c_double)]),
    "owqs_profile_run": (C.c_int, [C.c_void_p, C.POINTER(owqs_run_opts), C.c_void_p, C.c_void_p,
                                   C.POINTER(C.c_uint8), C.POINTER(C.c_float), C.POINTER(C.c_double),
                                   C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.c_uint32, C.POINTER(C.c_uint32)]),
    "owqs_get_index_map": (C.c_int, [C.c_void_p, C.c_uint32, C.POINTER(C.c_int32)]),
    "owqs_plan_memory": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint32, C.c_uint32, C.POINTER(C.c_uint8),
                                   C.c_void_p]),
    "owqs_last_sample_info": (C.c_int, [C.c_void_p, C.POINTER(owqs_sample_info)]),
    "owqs_describe_groups": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint32, C.c_uint32, C.POINTER(C.c_uint8),
                                       C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                       C.POINTER(C.c_uint32), C.c_uint32, C.POINTER(C.c_uint32)]),
    "owqs_describe_passes": (C.c_int, [C.c_void_p, C.c_uint32, C.POINTER(C.c_uint8), C.POINTER(owqs_pass_desc),
                                       C.c_uint32, C.POINTER(C.c_uint32)]),
    "owqs_reorder_features": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint32, C.POINTER(C.c_uint32), C.c_uint32,
                                        C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64,
                                        C.POINTER(C.c_uint64)]),
    "owqs_model_create": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(C.c_void_p)]),
    "owqs_model_free": (None, [C.c_void_p]),
    "owqs_model_get_weights": (C.c_int, [C.c_void_p, C.c_void_p]),
    "owqs_model_score": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p]),
    "owqs_model_gradient": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p,
                                      C.POINTER(C.c_float), C.c_void_p]),
    "owqs_model_train": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32, C.c_uint32,
                                   C.c_uint32, C.c_float, C.c_uint64, C.c_void_p, C.c_void_p]),
    "owqs_find_flow": (C.c_int, [C.c_void_p, C.c_uint32, C.POINTER(C.c_uint32), C.POINTER(C.c_int32),
                                 C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.c_uint32, C.POINTER(C.c_uint32)]),
    "owqs_test_wait_timeout": (C.c_int, [C.c_uint32, C.c_uint64]),
    "owqs_test_shrink_extents": (C.c_int, [C.c_uint32, C.c_uint64]),
    "owqs_test_grid_cap": (C.c_int, [C.c_uint32]),
    "owqs_test_group_m4_width": (C.c_int, [C.c_uint32]),
    "owqs_describe_launches": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint32, C.c_uint32, C.POINTER(C.c_uint8),
                                         C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                         C.c_uint32, C.POINTER(C.c_uint32)]),
    "owqs_run_product": (C.c_int, [C.c_void_p, C.POINTER(owqs_run_opts), C.c_uint32, C.POINTER(C.c_uint32),
                                   C.POINTER(C.c_uint32), C.POINTER(C.c_void_p), C.c_void_p, C.POINTER(C.c_uint8),
                                   C.POINTER(C.c_double)]),
    "owqs_last_error": (C.c_char_p, []),
    "owqs_abi_version": (C.c_uint32, []),
}

_lib = None


def library(path: str = LIB_PATH):
    """Load libowqs.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(st: int):
    if st != OK:
        raise OwqsError(st, library().owqs_last_error().decode())


def _check_vectors(psi_in, out, tdt, nin: int, nout: int, out_elems: Optional[int] = None):
    """The library takes raw device pointers and trusts their extents, so a
    wrongly sized, typed or placed tensor is refused here, before any call:
    psi_in (when given) must hold exactly 2^nin amplitudes, out at least
    2^nout (out_elems when given), both contiguous CUDA tensors of the run's
    dtype on one device."""
    if psi_in is not None:
        if not psi_in.is_cuda or psi_in.dtype != tdt or not psi_in.is_contiguous():
            raise ValueError("psi_in must be a contiguous CUDA tensor of the run's dtype")
        if psi_in.numel() != (1 << nin):
            raise ValueError(f"psi_in holds {psi_in.numel()} amplitudes; the pattern has {nin} input qubits "
                             f"(2^{nin} = {1 << nin} amplitudes)")
    if out is not None:
        need = (1 << nout) if out_elems is None else out_elems
        if not out.is_cuda or out.dtype != tdt or not out.is_contiguous():
            raise ValueError("out must be a contiguous CUDA tensor of the run's dtype")
        if out.numel() < need:
            raise ValueError(f"out holds {out.numel()} amplitudes; the run writes {need}")
        if psi_in is not None and out.device != psi_in.device:
            raise ValueError("psi_in and out must be on the same device")


def _check_host_vectors(psi_in, out, dtype: str, nin: int, nout: int):
    """run_host's counterpart of _check_vectors: numpy arrays or CPU torch
    tensors (pinned for full-speed copies) of the run's dtype, contiguous,
    psi_in exactly 2^nin amplitudes and out at least 2^nout."""
    ndt = np.complex64 if dtype == "c64" else np.complex128
    for name, a, n, exact in (("psi_in", psi_in, nin, True), ("out", out, nout, False)):
        if a is None:
            continue
        if isinstance(a, np.ndarray):
            ok = a.dtype == ndt and a.flags["C_CONTIGUOUS"] and (name != "out" or a.flags["WRITEABLE"])
            size = a.size
        elif hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
            import torch
            tdt = torch.complex64 if dtype == "c64" else torch.complex128
            ok = (not a.is_cuda) and a.dtype == tdt and a.is_contiguous()
            size = a.numel()
        else:
            ok, size = False, 0
        if not ok:
            raise ValueError(f"{name} must be a contiguous, writeable host array (numpy or CPU torch) of "
                             f"{np.dtype(ndt).name}")
        if (size != (1 << n)) if exact else (size < (1 << n)):
            raise ValueError(f"{name} holds {size} amplitudes; the run needs {1 << n}")


def _u32(a: Sequence[int]):
    arr = (C.c_uint32 * max(1, len(a)))(*a)
    return arr


class Handle:
    """A loaded pattern (owned by the library)."""

    def __init__(self, pattern):
        lib = library()
        self.pattern = pattern
        cmds = (owqs_cmd * max(1, len(pattern.cmds)))()
        domain = []
        for i, c in enumerate(pattern.cmds):
            x = cmds[i]
            x.kind = CMD_KIND[c.kind]
            x.q0 = c.q0
            x.q1 = c.q1 if c.kind == "E" else 0
            x.angle = c.angle
            x.s_off, x.s_len = len(domain), len(c.sdom)
            domain += list(c.sdom)
            x.t_off, x.t_len = len(domain), len(c.tdom)
            domain += list(c.tdom)
        h = C.c_void_p()
        _check(lib.owqs_load_pattern(pattern.nqubits, _u32(pattern.inputs), len(pattern.inputs),
                                     _u32(pattern.outputs), len(pattern.outputs), cmds, len(pattern.cmds),
                                     _u32(domain), len(domain), C.byref(h)))
        self._h = h
        self.K = sum(1 for c in pattern.cmds if c.kind == "M")
        self.nin = len(pattern.inputs)
        self.nout = len(pattern.outputs)

    def close(self):
        if getattr(self, "_h", None):
            library().owqs_free_pattern(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- host-only calls -------------------------------------------------
    def info(self) -> dict:
        i = owqs_pattern_info()
        _check(library().owqs_get_info(self._h, C.byref(i)))
        return {f: getattr(i, f) for f, _ in owqs_pattern_info._fields_}

    def reorder(self, mode: str = "owqs", product_input: bool = False, sweep: bool = True,
                weights=(1.0, 1.0, 0.5, 1.0), model=None):
        o = owqs_reorder_opts(MODE[mode], int(product_input), int(sweep), int(model is not None), *weights,
                              model._m if model is not None else None)
        info = owqs_reorder_info()
        order = (C.c_uint32 * max(1, self.K))()
        _check(library().owqs_reorder(self._h, C.byref(o), C.byref(info), order))
        return list(order)[: self.K], {f: getattr(info, f) for f, _ in owqs_reorder_info._fields_ if f != "pad_"}

    def set_order(self, order: Sequence[int]):
        _check(library().owqs_set_order(self._h, _u32(order), len(order)))

    def reset_order(self):
        _check(library().owqs_reset_order(self._h))

    def order(self):
        out = (C.c_uint32 * max(1, self.K))()
        _check(library().owqs_get_order(self._h, out))
        return list(out)[: self.K]

    def features(self, order, mode: str = "eowqs", product_input: bool = False, max_cands: int = 32,
                 seed: int = 0):
        """Training rows along `order`: (feats [rows, F] float32, step_first
        [K+1] uint32, target_row [K] uint32)."""
        ordr = _u32(order)
        n = C.c_uint64()
        st = library().owqs_reorder_features(self._h, MODE[mode], int(product_input), ordr, max_cands, seed,
                                             None, None, None, 0, C.byref(n))
        if st not in (OK, ERR_ARG):
            _check(st)
        feats = np.zeros((max(1, n.value), NFEAT), dtype=np.float32)
        first = np.zeros(self.K + 1, dtype=np.uint32)
        tgt = np.zeros(max(1, self.K), dtype=np.uint32)
        _check(library().owqs_reorder_features(self._h, MODE[mode], int(product_input), ordr, max_cands, seed,
                                               feats.ctypes.data, first.ctypes.data, tgt.ctypes.data, n.value,
                                               C.byref(n)))
        return feats[: n.value], first, tgt[: self.K]

    def find_flow(self, kind: str = "gflow"):
        """Flow of the open graph (kind "causal" or "gflow"): None if there is
        none, else (layer per label, g per measured label as a sorted list)."""
        k = {"causal": FLOW_CAUSAL, "gflow": FLOW_GFLOW}[kind]
        n = self.pattern.nqubits
        found, total = C.c_uint32(), C.c_uint32()
        layer = (C.c_int32 * n)()
        first = (C.c_uint32 * (n + 1))()
        _check(library().owqs_find_flow(self._h, k, C.byref(found), layer, first, None, 0, C.byref(total)))
        if not found.value:
            return None
        members = (C.c_uint32 * max(1, total.value))()
        _check(library().owqs_find_flow(self._h, k, C.byref(found), layer, first, members, total.value,
                                        C.byref(total)))
        outs = set(self.pattern.outputs)
        g = {v: list(members[first[v]:first[v + 1]]) for v in range(n) if v not in outs}
        return list(layer), g

    def describe_launches(self, outcomes=None, *, dtype: str = "c64", mode: str = "owqs", real_input: bool = False):
        """The launches a run would make (host only): list of (kind name,
        first measurement, measurements)."""
        cap = 2 * self.K + 16
        kd = (C.c_uint32 * cap)()
        fm = (C.c_uint32 * cap)()
        nm = (C.c_uint32 * cap)()
        n = C.c_uint32()
        oc = _outcome_buf(outcomes, self.K) if outcomes is not None else None
        _check(library().owqs_describe_launches(self._h, DTYPE[dtype], MODE[mode], int(real_input), oc, kd, fm, nm,
                                                cap, C.byref(n)))
        return [(KERNEL_KIND[kd[i]], fm[i], nm[i]) for i in range(min(n.value, cap))]

    def plan_memory(self, outcomes=None, *, dtype: str = "c64", mode: str = "owqs", real_input: bool = False):
        """One live array against separate sub-states for the active order
        (host only): the paper's m, components, joins, arena and one-array
        bytes, and which a default run takes."""
        plan = owqs_memory_plan()
        oc = _outcome_buf(outcomes, self.K) if outcomes is not None else None
        _check(library().owqs_plan_memory(self._h, DTYPE[dtype], MODE[mode], int(real_input), oc, C.byref(plan)))
        return {f: getattr(plan, f) for f, _ in owqs_memory_plan._fields_}

    def last_sample_info(self):
        """How the last sampled run was carried out: path ("guess_kept",
        "checked_launches", "one_at_a_time", ...), whether a whole-run guess
        ran first, host checks and relaunches of checked launches."""
        info = owqs_sample_info()
        _check(library().owqs_last_sample_info(self._h, C.byref(info)))
        return {"path": SAMPLE_PATH.get(info.path, str(info.path)), "guessed": bool(info.guessed),
                "checks": info.checks, "relaunches": info.relaunches}

    def describe_groups(self, outcomes=None, *, dtype: str = "c64", mode: str = "owqs", real_input: bool = False):
        """The pass groups a run would launch (host only): list of dicts with
        the register qubits m, the slot sequence, whether every probability
        of the group is exactly 1/2 (half), the input width n_in and whether
        a kernel compiled for that sequence runs it."""
        cap = self.K + 16
        regs, slots, nin, spec = ((C.c_uint32 * cap)() for _ in range(4))
        n = C.c_uint32()
        oc = _outcome_buf(outcomes, self.K) if outcomes is not None else None
        _check(library().owqs_describe_groups(self._h, DTYPE[dtype], MODE[mode], int(real_input), oc, regs, slots,
                                              nin, spec, cap, C.byref(n)))
        out = []
        for i in range(min(n.value, cap)):
            k = (slots[i] >> 24) & 15
            out.append({"m": regs[i], "slots": tuple((slots[i] >> (2 * j)) & 3 for j in range(k)),
                        "half": bool((slots[i] >> 31) & 1), "n_in": nin[i], "specialised": bool(spec[i])})
        return out

    def index_map(self, pass_index: int):
        out = (C.c_int32 * self.pattern.nqubits)()
        _check(library().owqs_get_index_map(self._h, pass_index, out))
        return list(out)

    def describe_passes(self, outcomes=None, mode: str = "owqs"):
        n = C.c_uint32()
        oc = _outcome_buf(outcomes, self.K)
        _check(library().owqs_describe_passes(self._h, MODE[mode], oc, None, 0, C.byref(n)))
        buf = (owqs_pass_desc * max(1, n.value))()
        _check(library().owqs_describe_passes(self._h, MODE[mode], oc, buf, n.value, C.byref(n)))
        return [buf[i] for i in range(n.value)]

    # -- device calls ----------------------------------------------------
    def run(self, psi_in=None, *, dtype: str = "c128", mode: str = "owqs", policy: str = "forced",
            outcomes=None, seed: int = 0, stream=None, use_graph: bool = True, out=None,
            check: bool = True, host_sampling: bool = False, per_pass: bool = False,
            sequential_sampling: bool = False, layout: str = "auto", double_float: bool = False):
        """Run on the GPU.  psi_in: torch tensor on the GPU (complex64 for
        c64, complex128 for c128) or None for |+> inputs; returns
        (psi_out tensor, outcomes array, probs array, status).
        host_sampling: draw sampled outcomes on the host (one device read per
        measurement) instead of on the device.  per_pass: one kernel per pass
        even for a run that fits the single-block kernel.
        sequential_sampling: draw sampled OWQS outcomes one measurement at a
        time from the start, instead of first checking the guess u > 1/2 with
        one forced run.
        layout: "auto" (separate sub-states when they need at most half the
        memory of one array), "substates" or "one_array".
        double_float: complex128 pass groups in double-float arithmetic on the
        FP32 pipes."""
        import torch
        tdt = torch.complex64 if dtype == "c64" else torch.complex128
        _check_vectors(psi_in, out, tdt, self.nin, self.nout)
        dev = psi_in.device if psi_in is not None else torch.device("cuda", torch.cuda.current_device())
        if out is None:
            out = torch.empty(1 << self.nout, dtype=tdt, device=dev)
        oc = np.zeros(max(1, self.K), dtype=np.uint8)
        if outcomes is not None:
            oc[: self.K] = np.asarray(outcomes, dtype=np.uint8)[: self.K]
        probs = np.zeros(max(1, self.K), dtype=np.float64)
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        opts = owqs_run_opts(DTYPE[dtype], MODE[mode], POLICY[policy], 0, seed, C.c_void_p(s.cuda_stream),
                             int(use_graph), (RUN_HOST_SAMPLING if host_sampling else 0) |
                             (RUN_PER_PASS if per_pass else 0) |
                             (RUN_SEQUENTIAL_SAMPLING if sequential_sampling else 0) |
                             {"auto": 0, "substates": RUN_SUBSTATES, "one_array": RUN_ONE_ARRAY}[layout] |
                             (RUN_DOUBLE_FLOAT if double_float else 0))
        st = library().owqs_run(self._h, C.byref(opts), C.c_void_p(psi_in.data_ptr() if psi_in is not None else 0),
                                C.c_void_p(out.data_ptr()), oc.ctypes.data_as(C.POINTER(C.c_uint8)),
                                probs.ctypes.data_as(C.POINTER(C.c_double)))
        if check and st not in (OK,):
            _check(st)
        return out, oc[: self.K].copy(), probs[: self.K].copy(), st

    def run_async(self, psi_in, out, *, dtype: str = "c64", mode: str = "owqs", policy: str = "forced",
                  outcomes=None, stream=None, double_float: bool = False):
        """owqs_run_async: enqueue a run and return.  psi_in (or None for |+>)
        and out: CUDA tensors, or pinned CPU tensors / numpy arrays (host
        vectors, copied on the library's copy streams).  They must stay alive
        and out unread until wait() has returned for this run."""
        import torch
        host = not (isinstance(out, torch.Tensor) and out.is_cuda)
        if host:
            _check_host_vectors(psi_in, out, dtype, self.nin, self.nout)
            pin = 0 if psi_in is None else _host_ptr(psi_in)
            pout = _host_ptr(out)
            dev = torch.device("cuda", torch.cuda.current_device())
        else:
            tdt = torch.complex64 if dtype == "c64" else torch.complex128
            _check_vectors(psi_in, out, tdt, self.nin, self.nout)
            pin = 0 if psi_in is None else psi_in.data_ptr()
            pout = out.data_ptr()
            dev = out.device
        oc = np.zeros(max(1, self.K), dtype=np.uint8)
        if outcomes is not None:
            oc[: self.K] = np.asarray(outcomes, dtype=np.uint8)[: self.K]
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        opts = owqs_run_opts(DTYPE[dtype], MODE[mode], POLICY[policy], 1 if host else 0, 0,
                             C.c_void_p(s.cuda_stream), 0, RUN_DOUBLE_FLOAT if double_float else 0)
        _check(library().owqs_run_async(self._h, C.byref(opts), C.c_void_p(pin), C.c_void_p(pout),
                                        oc.ctypes.data_as(C.POINTER(C.c_uint8))))

    def wait(self, check: bool = True):
        """owqs_wait: finish the oldest run in flight; returns (outcomes,
        probs, status)."""
        oc = np.zeros(max(1, self.K), dtype=np.uint8)
        probs = np.zeros(max(1, self.K), dtype=np.float64)
        st = library().owqs_wait(self._h, oc.ctypes.data_as(C.POINTER(C.c_uint8)),
                                 probs.ctypes.data_as(C.POINTER(C.c_double)))
        if check and st != OK:
            _check(st)
        return oc[: self.K].copy(), probs[: self.K].copy(), st

    def run_product(self, factors, *, dtype: str = "c128", mode: str = "owqs", policy: str = "forced",
                    outcomes=None, stream=None, use_graph: bool = True, out=None, check: bool = True):
        """Run with a product input: factors is a list of (qubits, CUDA
        tensor) pairs, tensor bit k = qubits[k]; returns as run()."""
        import torch
        tdt = torch.complex64 if dtype == "c64" else torch.complex128
        sizes, qubits, vecs = [], [], []
        for qs, v in factors:
            if not v.is_cuda or v.dtype != tdt or not v.is_contiguous() or v.numel() != (1 << len(qs)):
                raise ValueError("each factor must be a contiguous CUDA tensor of the run's dtype, 2^len(qubits) long")
            sizes.append(len(qs))
            qubits += list(qs)
            vecs.append(v.data_ptr())
        dev = factors[0][1].device if factors else torch.device("cuda", torch.cuda.current_device())
        _check_vectors(None, out, tdt, 0, self.nout)
        if out is None:
            out = torch.empty(1 << self.nout, dtype=tdt, device=dev)
        oc = np.zeros(max(1, self.K), dtype=np.uint8)
        if outcomes is not None:
            oc[: self.K] = np.asarray(outcomes, dtype=np.uint8)[: self.K]
        probs = np.zeros(max(1, self.K), dtype=np.float64)
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        opts = owqs_run_opts(DTYPE[dtype], MODE[mode], POLICY[policy], 0, 0, C.c_void_p(s.cuda_stream),
                             int(use_graph), 0)
        vp = (C.c_void_p * max(1, len(vecs)))(*vecs)
        st = library().owqs_run_product(self._h, C.byref(opts), len(sizes), _u32(sizes), _u32(qubits), vp,
                                        C.c_void_p(out.data_ptr()), oc.ctypes.data_as(C.POINTER(C.c_uint8)),
                                        probs.ctypes.data_as(C.POINTER(C.c_double)))
        if check and st != OK:
            _check(st)
        return out, oc[: self.K].copy(), probs[: self.K].copy(), st

    def unitary(self, *, dtype: str = "c128", outcomes=None, stream=None, use_graph: bool = True, out=None,
                per_pass: bool = False):
        """All basis columns of the forced branch as a matrix (2^|O| x 2^|I|,
        column-major as a flat tensor); returns (U, ||U||_F^2 / 2^|I|)."""
        import torch
        tdt = torch.complex64 if dtype == "c64" else torch.complex128
        _check_vectors(None, out, tdt, 0, self.nout + self.nin)
        if out is None:
            out = torch.empty(1 << (self.nout + self.nin), dtype=tdt, device="cuda")
        s = stream if stream is not None else torch.cuda.current_stream()
        policy = "zero" if outcomes is None else "forced"
        opts = owqs_run_opts(DTYPE[dtype], MODE["eowqs"], POLICY[policy], 0, 0, C.c_void_p(s.cuda_stream),
                             int(use_graph), RUN_PER_PASS if per_pass else 0)
        f2 = C.c_double()
        _check(library().owqs_unitary(self._h, C.byref(opts), _outcome_buf(outcomes, self.K),
                                      C.c_void_p(out.data_ptr()), C.byref(f2)))
        return out, f2.value

    def run_static(self, psi_in=None, *, dtype: str = "c128", mode: str = "owqs", policy: str = "forced",
                   outcomes=None, stream=None, out=None, check: bool = True):
        """owqs_run_static: same as run() without any device allocation inside
        the library (scratch in a fixed device array; small patterns only)."""
        import torch
        tdt = torch.complex64 if dtype == "c64" else torch.complex128
        _check_vectors(psi_in, out, tdt, self.nin, self.nout)
        dev = psi_in.device if psi_in is not None else torch.device("cuda", torch.cuda.current_device())
        if out is None:
            out = torch.empty(1 << self.nout, dtype=tdt, device=dev)
        oc = np.zeros(max(1, self.K), dtype=np.uint8)
        if outcomes is not None:
            oc[: self.K] = np.asarray(outcomes, dtype=np.uint8)[: self.K]
        probs = np.zeros(max(1, self.K), dtype=np.float64)
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        opts = owqs_run_opts(DTYPE[dtype], MODE[mode], POLICY[policy], 0, 0, C.c_void_p(s.cuda_stream), 0, 0)
        st = library().owqs_run_static(self._h, C.byref(opts),
                                       C.c_void_p(psi_in.data_ptr() if psi_in is not None else 0),
                                       C.c_void_p(out.data_ptr()), oc.ctypes.data_as(C.POINTER(C.c_uint8)),
                                       probs.ctypes.data_as(C.POINTER(C.c_double)))
        if check and st != OK:
            _check(st)
        return out, oc[: self.K].copy(), probs[: self.K].copy(), st

    def run_host(self, psi_in: Optional[np.ndarray], out: np.ndarray, *, dtype: str = "c64",
                 mode: str = "owqs", policy: str = "forced", outcomes=None, seed: int = 0, stream=None,
                 use_graph: bool = True):
        """Run with host vectors; the library copies them in and out."""
        import torch
        _check_host_vectors(psi_in, out, dtype, self.nin, self.nout)
        oc = np.zeros(max(1, self.K), dtype=np.uint8)
        if outcomes is not None:
            oc[: self.K] = np.asarray(outcomes, dtype=np.uint8)[: self.K]
        probs = np.zeros(max(1, self.K), dtype=np.float64)
        s = stream if stream is not None else torch.cuda.current_stream()
        opts = owqs_run_opts(DTYPE[dtype], MODE[mode], POLICY[policy], 1, seed, C.c_void_p(s.cuda_stream),
                             int(use_graph), 0)
        pin = 0 if psi_in is None else _host_ptr(psi_in)
        _check(library().owqs_run(self._h, C.byref(opts), C.c_void_p(pin), C.c_void_p(_host_ptr(out)),
                                  oc.ctypes.data_as(C.POINTER(C.c_uint8)),
                                  probs.ctypes.data_as(C.POINTER(C.c_double))))
        return oc[: self.K].copy(), probs[: self.K].copy()

    def profile(self, psi_in=None, *, dtype: str = "c64", mode: str = "owqs", policy: str = "forced",
                outcomes=None, stream=None, out=None, layout: str = "auto", double_float: bool = False):
        """Per-launch CUDA-event durations of one run (no graph)."""
        import torch
        tdt = torch.complex64 if dtype == "c64" else torch.complex128
        _check_vectors(psi_in, out, tdt, self.nin, self.nout)
        dev = torch.device("cuda", torch.cuda.current_device())
        if out is None:
            out = torch.empty(1 << self.nout, dtype=tdt, device=dev)
        cap = 4 * self.K + 16
        ms = (C.c_float * cap)()
        by = (C.c_double * cap)()
        kd = (C.c_uint32 * cap)()
        nm = (C.c_uint32 * cap)()
        n = C.c_uint32()
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        opts = owqs_run_opts(DTYPE[dtype], MODE[mode], POLICY[policy], 0, 0, C.c_void_p(s.cuda_stream), 0,
                             {"auto": 0, "substates": RUN_SUBSTATES, "one_array": RUN_ONE_ARRAY}[layout] |
                             (RUN_DOUBLE_FLOAT if double_float else 0))
        oc = _outcome_buf(outcomes, self.K)
        _check(library().owqs_profile_run(self._h, C.byref(opts),
                                          C.c_void_p(psi_in.data_ptr() if psi_in is not None else 0),
                                          C.c_void_p(out.data_ptr()), oc, ms, by, kd, nm, cap, C.byref(n)))
        k = min(n.value, cap)
        self.profile_meas = np.array(nm[:k])  # measurements per launch of the last profile
        return np.array(ms[:k]), np.array(by[:k]), np.array(kd[:k]), out


def last_error() -> str:
    """Message of the library's last error on this thread."""
    return library().owqs_last_error().decode()


def test_wait_timeout(runs: int, limit_cycles: int = 2_000_000):
    """Make the next `runs` runs give up on a device-side wait (test hook)."""
    _check(library().owqs_test_wait_timeout(runs, limit_cycles))


def test_grid_cap(blocks: int):
    """Cap every later pass-kernel launch at `blocks` thread blocks (test
    hook; 0 removes the cap), so that small arrays make the persistent
    kernels loop over many tiles per warp."""
    _check(library().owqs_test_grid_cap(int(blocks)))


def test_group_m4_width(width: int):
    """Let complex64 pass groups take a 4-qubit register from input width
    `width` on (test hook; 0 restores the default)."""
    _check(library().owqs_test_group_m4_width(int(width)))


def test_shrink_extents(runs: int, elems: int):
    """Make the next `runs` runs carry buffer extents `elems` amplitudes short
    (test hook; only the bounds-checked build reads them)."""
    _check(library().owqs_test_shrink_extents(runs, elems))


def run_batch(items, *, dtype: str = "c128", column_block: int = 0, stream=None, use_graph: bool = True,
              overlaps: bool = False):
    """owqs_run_batch.  items: list of dicts with keys handle, outcomes (array
    or None), psi_in (CUDA tensor or None), out (CUDA tensor), ref (int, -1).
    Returns (info dict, overlaps array of shape (n, 4) or None)."""
    import torch
    n = len(items)
    # the item structs as one numpy record array (the layout of
    # owqs_batch_item) and every item's outcomes in one byte buffer
    rec = np.zeros(max(1, n), dtype=_BATCH_ITEM_DTYPE)
    ks = np.array([max(1, it["handle"].K) for it in items], dtype=np.int64)
    offs = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(ks, out=offs[1:])
    ocbuf = np.zeros(max(1, int(offs[-1])), dtype=np.uint8)
    base = ocbuf.ctypes.data
    pat, ocp, pin, pout, ref = (np.zeros(n, dtype=np.uint64), np.zeros(n, dtype=np.uint64),
                                np.zeros(n, dtype=np.uint64), np.zeros(n, dtype=np.uint64),
                                np.zeros(n, dtype=np.int32))
    for i, it in enumerate(items):
        h = it["handle"]
        oc = it.get("outcomes")
        if oc is not None:
            a = np.asarray(oc).ravel()[: h.K]
            ocbuf[offs[i]: offs[i] + a.size] = a.astype(np.uint8) & 1
            ocp[i] = base + int(offs[i])
        pat[i] = h._h.value
        x = it.get("psi_in")
        if x is not None:
            pin[i] = x.data_ptr()
        pout[i] = it["out"].data_ptr()
        ref[i] = int(it.get("ref", -1))
    if n:
        rec["pattern"][:n], rec["outcomes"][:n], rec["psi_in"][:n], rec["out"][:n] = pat, ocp, pin, pout
        rec["ref"][:n] = ref
    arr = rec.ctypes.data_as(C.POINTER(owqs_batch_item))
    ov = np.zeros(4 * max(1, n), dtype=np.float64) if overlaps else None
    s = stream if stream is not None else torch.cuda.current_stream()
    opts = owqs_batch_opts(DTYPE[dtype], column_block, C.c_void_p(s.cuda_stream), int(use_graph), 0,
                           ov.ctypes.data_as(C.POINTER(C.c_double)) if ov is not None else None)
    info = owqs_batch_info()
    _check(library().owqs_run_batch(arr, n, C.byref(opts), C.byref(info)))
    return ({f: getattr(info, f) for f, _ in owqs_batch_info._fields_ if f != "pad_"},
            ov[: 4 * n].reshape(n, 4) if ov is not None else None)


NFEAT = 12
NPARAM = 5057


class Model:
    """The learned reorder proposal's network (device resident)."""

    def __init__(self, weights: Optional[np.ndarray] = None, seed: int = 0):
        lib = library()
        m = C.c_void_p()
        if weights is not None:
            w = np.ascontiguousarray(weights, dtype=np.float32)
            if w.size != NPARAM:
                raise ValueError(f"expected {NPARAM} weights")
            _check(lib.owqs_model_create(w.ctypes.data, seed, C.byref(m)))
        else:
            _check(lib.owqs_model_create(None, seed, C.byref(m)))
        self._m = m

    def close(self):
        if getattr(self, "_m", None):
            library().owqs_model_free(self._m)
            self._m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def weights(self) -> np.ndarray:
        w = np.zeros(NPARAM, dtype=np.float32)
        _check(library().owqs_model_get_weights(self._m, w.ctypes.data))
        return w

    def score(self, feats_dev, stream=None):
        import torch
        out = torch.empty(feats_dev.shape[0], dtype=torch.float32, device=feats_dev.device)
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(library().owqs_model_score(self._m, feats_dev.data_ptr(), feats_dev.shape[0], out.data_ptr(),
                                          C.c_void_p(s.cuda_stream)))
        return out

    def gradient(self, feats_dev, first_dev, target_dev, stream=None):
        import torch
        g = np.zeros(NPARAM, dtype=np.float32)
        loss = C.c_float()
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(library().owqs_model_gradient(self._m, feats_dev.data_ptr(), first_dev.data_ptr(),
                                             target_dev.data_ptr(), target_dev.shape[0], g.ctypes.data,
                                             C.byref(loss), C.c_void_p(s.cuda_stream)))
        return g, loss.value

    def train(self, feats_dev, first_dev, target_dev, *, epochs: int = 10, batch_steps: int = 512,
              lr: float = 1e-3, seed: int = 0, stream=None):
        import torch
        losses = np.zeros(max(1, epochs), dtype=np.float32)
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(library().owqs_model_train(self._m, feats_dev.data_ptr(), first_dev.data_ptr(),
                                          target_dev.data_ptr(), target_dev.shape[0], epochs, batch_steps, lr,
                                          seed, losses.ctypes.data, C.c_void_p(s.cuda_stream)))
        return losses[:epochs]


def _host_ptr(a) -> int:
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _outcome_buf(outcomes, K):
    if outcomes is None:
        return None
    arr = (C.c_uint8 * max(1, K))(*[int(x) & 1 for x in list(outcomes)[:K]])
    return arr


def load(pattern) -> Handle:
    return Handle(pattern)
