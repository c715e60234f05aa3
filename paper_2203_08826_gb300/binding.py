"""Thin ctypes binding of libqsim (argument marshalling only).

Every function here forwards to the C ABI declared in ``include/qsim.h``;
no simulation arithmetic happens in Python.  PyTorch supplies device memory
(state tensors) and the CUDA stream (``torch.cuda.current_stream()``).
The library must have been built (``paper_2203_08826_gb300.build.build()``);
loading raises ``QsimError`` otherwise -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Iterable, Sequence

import numpy as np

from . import inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
# QSIM_LIBRARY=debug loads the build with index bound checks (build(debug=True))
LIB_PATH = (os.path.join(_HERE, "_build_debug", "libqsim_debug.so") if os.environ.get("QSIM_LIBRARY") == "debug"
            else os.path.join(_HERE, "_build", "libqsim.so"))

C64, C128 = 0, 1
FUSE_GREEDY2, FUSE_STAGED, FUSE_TC = 0, 1, 2
SPECIALIZE = 0x100  # ORed into FUSE_STAGED: stage kernels compiled for the plan
PREC_BF16X3, PREC_TF32X3, PREC_FP32 = 0, 1, 2
INIT_ZERO, INIT_BASIS, INIT_HOST, INIT_DEVICE, INIT_NULL = 0, 1, 2, 3, 4
SLICE_SEGMENT, SLICE_SWAP = 0, 1
SLICES_DEVICE, SLICES_HOST = 0, 1
GATE_KIND = {"matrix": 0, "h": 1, "x": 2, "y": 3, "z": 4, "s": 5, "t": 6, "rx": 7, "ry": 8,
             "rz": 9, "phase": 10, "cz": 11, "swap": 12, "su2": 13, "rzz": 14}


class QsimError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"qsim error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None

P, I, U64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_double
_SIGS = {
    "qsim_last_error": ([], ctypes.c_char_p),
    "qsim_version": ([], ctypes.c_char_p),
    "qsim_state_create": ([I, I, P, P, P], I),
    "qsim_state_destroy": ([P], I),
    "qsim_state_set_stream": ([P, P], I),
    "qsim_state_info": ([P, P, P, P], I),
    "qsim_state_init": ([P, I, U64, P], I),
    "qsim_state_copy_to_host": ([P, P], I),
    "qsim_synchronize": ([P], I),
    "qsim_apply_gate": ([P, P, P, I, P, I], I),
    "qsim_apply_named": ([P, I, P, I, P, I, P], I),
    "qsim_circuit_create": ([I, P], I),
    "qsim_circuit_destroy": ([P], I),
    "qsim_circuit_add": ([P, I, P, I, P, I, P, I, P], I),
    "qsim_circuit_info": ([P, P, P, P], I),
    "qsim_circuit_gate": ([P, I, P, P, P, P, P, P], I),
    "qsim_run": ([P, P], I),
    "qsim_plan_build": ([P, I, I, P], I),
    "qsim_plan_destroy": ([P], I),
    "qsim_plan_info": ([P, P, P, P], I),
    "qsim_plan_block": ([P, I, P, P, P], I),
    "qsim_plan_describe": ([P, P, ctypes.c_size_t], I),
    "qsim_plan_source": ([P, I, P, ctypes.c_size_t, P], I),
    "qsim_plan_stage_dump": ([P, I, P, ctypes.c_size_t, P], I),
    "qsim_spec_stats": ([P, P, P], I),
    "qsim_plan_flops": ([P, P, P], I),
    "qsim_adjoint_specialize": ([I, P], I),
    "qsim_plan_tc_pass": ([P, I, P, P, P, P, P, P, P], I),
    "qsim_plan_tc_epilogue": ([P, I, I, P, P, P, P, P], I),
    "qsim_plan_stage": ([P, I, P, P, P, P, P], I),
    "qsim_plan_tc_precision": ([P, I, P], I),
    "qsim_plan_tc_set_precision": ([P, I, P], I),
    "qsim_apply_fused": ([P, P], I),
    "qsim_plan_autotune": ([P, P, I, P, P, P, P], I),
    "qsim_plan_autotune_ex": ([P, P, I, D, P, P, I, P], I),
    "qsim_probabilities": ([P, P, I, P, I], I),
    "qsim_norm2": ([P, P], I),
    "qsim_sample": ([P, U64, U64, U64, P, I], I),
    "qsim_sample_probs": ([P, U64, U64, U64, U64, P, I, P], I),
    "qsim_sample_probs_static": ([P, U64, U64, U64, U64, P, P], I),
    "qsim_expectation_pauli": ([P, I, P, P, P, P], I),
    "qsim_collapse": ([P, P, I, U64, P], I),
    "qsim_adjoint_grad": ([P, P, I, I, P, I, P, P, P, P, P, P], I),
    "qsim_batch_create": ([I, P, P], I),
    "qsim_batch_destroy": ([P], I),
    "qsim_batch_run": ([P, P, P], I),
    "qsim_batch_set_config": ([P, I, I], I),
    "qsim_batch_autotune": ([P, P, I, P, P, P], I),
    "qsim_apply_pauli_phase": ([P, I, P, P, D], I),
    "qsim_slice_plan_build": ([P, I, I, I, I, P], I),
    "qsim_slice_plan_destroy": ([P], I),
    "qsim_slice_plan_info": ([P, P, P, P, P, P], I),
    "qsim_slice_plan_step": ([P, I, P, P, P, P, P], I),
    "qsim_slice_plan_layout": ([P, P], I),
    "qsim_slice_segment_circuit": ([P, I, ctypes.c_uint32, P], I),
    "qsim_slice_apply_segment": ([P, I, ctypes.c_uint32, P], I),
    "qsim_slice_exchange": ([P, P, I, I, I, P], I),
    "qsim_slice_pack": ([P, I, I, I, I, P, P], I),
    "qsim_slice_unpack": ([P, I, I, I, I, P, P], I),
    "qsim_slice_run": ([P, I, P, I, P], I),
    "qsim_sampler_weight_c64": ([ctypes.c_float, ctypes.c_float], U64),
    "qsim_prob_c64": ([ctypes.c_float, ctypes.c_float], D),
    "qsim_debug_fail_alloc": ([I, I], I),
    "qsim_debug_set_wait_limit": ([ctypes.c_ulonglong], I),
    "qsim_debug_checks": ([I], ctypes.c_longlong),
    "qsim_profile_enable": ([I], I),
    "qsim_profile_reset": ([], I),
    "qsim_profile_count": ([P], I),
    "qsim_profile_get": ([I, P, P, P, P, P], I),
    "qsim_launch_count": ([], U64),
}


def lib():
    """The loaded libqsim (raises QsimError if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise QsimError(-5, f"{LIB_PATH} not built; run paper_2203_08826_gb300.build.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in _SIGS.items():
                f = getattr(L, name, None)
                if f is None:
                    continue
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise QsimError(rc, lib().qsim_last_error().decode())


def _arr(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None and a.size else None


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# ------------------------------------------------------------------ circuits
class QCircuit:
    """A circuit handle in the library, built from an ``inputs.Circuit``."""

    def __init__(self, circuit: inputs.Circuit):
        self.n = circuit.n
        self.source = circuit
        h = ctypes.c_void_p()
        _check(lib().qsim_circuit_create(circuit.n, ctypes.byref(h)))
        self.handle = h
        for g in circuit.gates:
            t = _arr(g.targets, np.int32)
            c = _arr(g.controls if len(g.controls) else [0], np.int32)
            prm = _arr(list(g.params) + [0.0] * (4 - len(g.params)) if g.name != "matrix" else [0.0] * 4,
                       np.float64)
            mat = None
            if g.name == "matrix":
                mat = _arr(np.asarray(g.matrix, dtype=np.complex128).view(np.float64), np.float64)
            _check(lib().qsim_circuit_add(h, GATE_KIND[g.name], _p(t), len(g.targets),
                                          _p(c) if len(g.controls) else None, len(g.controls),
                                          _p(prm), g.pindex, _p(mat) if mat is not None else None))

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.qsim_circuit_destroy(self.handle)
            self.handle = None

    @property
    def ngates(self) -> int:
        n = ctypes.c_int(); g = ctypes.c_int(); p = ctypes.c_int()
        _check(lib().qsim_circuit_info(self.handle, ctypes.byref(n), ctypes.byref(g), ctypes.byref(p)))
        return g.value

    @property
    def nparams(self) -> int:
        n = ctypes.c_int(); g = ctypes.c_int(); p = ctypes.c_int()
        _check(lib().qsim_circuit_info(self.handle, ctypes.byref(n), ctypes.byref(g), ctypes.byref(p)))
        return p.value


def circuit_gates(handle) -> list:
    """The gates stored in a library circuit, as ``inputs.Gate`` matrix gates."""
    n, ng, npar = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().qsim_circuit_info(handle, ctypes.byref(n), ctypes.byref(ng), ctypes.byref(npar)))
    out = []
    for i in range(ng.value):
        k, nc = ctypes.c_int(), ctypes.c_int()
        _check(lib().qsim_circuit_gate(handle, i, None, ctypes.byref(k), None, ctypes.byref(nc), None, None))
        t = np.zeros(max(1, k.value), dtype=np.int32)
        c = np.zeros(max(1, nc.value), dtype=np.int32)
        m = np.zeros(2 * (1 << (2 * k.value)), dtype=np.float64)
        _check(lib().qsim_circuit_gate(handle, i, None, ctypes.byref(k), _p(t), ctypes.byref(nc), _p(c), _p(m)))
        d = 1 << k.value
        out.append(inputs.Gate("matrix", tuple(int(v) for v in t[: k.value]), tuple(int(v) for v in c[: nc.value]),
                               (), -1, m.view(np.complex128).reshape(d, d).copy()))
    return out


class _TuneEntry(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("kmax", ctypes.c_int), ("ms", ctypes.c_double), ("err", ctypes.c_double),
                ("max_abs", ctypes.c_double), ("ref", ctypes.c_int), ("npasses", ctypes.c_int),
                ("nfp32", ctypes.c_int)]


class Plan:
    """A fusion plan (QSIM_FUSE_GREEDY2 / STAGED / TC) built on the host."""

    def __init__(self, circuit, kmax: int = 2, mode: int = FUSE_GREEDY2):
        qc = circuit if isinstance(circuit, QCircuit) else QCircuit(circuit)
        self.n = qc.n
        h = ctypes.c_void_p()
        _check(lib().qsim_plan_build(qc.handle, kmax, mode, ctypes.byref(h)))
        self.handle = h
        self.mode = mode

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.qsim_plan_destroy(self.handle)
            self.handle = None

    @classmethod
    def autotune(cls, circuit, scratch_state: "State", reps: int = 1, max_err: float | None = None) -> "Plan":
        """Fastest plan for `circuit`, timed on `scratch_state` (overwritten).

        With `max_err`, every candidate's error is measured against the
        gate-by-gate complex128 run (or, when that does not fit, the FP32
        staged plan) by qsim_plan_autotune_ex, only plans within it qualify,
        and a tensor-core plan with FP32 passes mixed in may be added; the
        measured table is kept in `.table` (`ref`: 1 for the complex128
        reference; `npasses`, `nfp32`: tensor-core passes and how many run in
        FP32)."""
        qc = circuit if isinstance(circuit, QCircuit) else QCircuit(circuit)
        if max_err is not None:
            tab = (_TuneEntry * 16)()
            nt = ctypes.c_int()
            h = ctypes.c_void_p()
            _check(lib().qsim_plan_autotune_ex(qc.handle, scratch_state.handle, reps, float(max_err),
                                               ctypes.byref(h), tab, 16, ctypes.byref(nt)))
            self = cls.__new__(cls)
            info = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
            self.n, self.handle = qc.n, h
            _check(lib().qsim_plan_info(h, *[ctypes.byref(x) for x in info]))
            self.mode = info[2].value
            names = {FUSE_GREEDY2: "greedy2", FUSE_STAGED: "staged", FUSE_TC: "tc",
                     FUSE_STAGED | SPECIALIZE: "staged-spec"}
            self.table = [{"mode": names.get(e.mode, e.mode), "kmax": e.kmax, "ms": e.ms, "err": e.err,
                           "max_abs": e.max_abs, "ref": "fp64" if e.ref else "first candidate",
                           "npasses": e.npasses, "nfp32": e.nfp32} for e in tab[: nt.value]]
            ok = [e for e in self.table if e["ms"] >= 0 and 0 <= e["err"] <= max_err]
            best = min(ok, key=lambda e: e["ms"]) if ok else None
            self.kmax = best["kmax"] if best else 0
            self.nfp32 = best["nfp32"] if best else 0
            self.tuned_ms = best["ms"] if best else -1.0
            return self
        h = ctypes.c_void_p()
        mode, kmax, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(lib().qsim_plan_autotune(qc.handle, scratch_state.handle, reps, ctypes.byref(h),
                                        ctypes.byref(mode), ctypes.byref(kmax), ctypes.byref(ms)))
        self = cls.__new__(cls)
        self.n, self.handle, self.mode = qc.n, h, mode.value
        self.kmax, self.tuned_ms = kmax.value, ms.value
        return self

    def tc_precisions(self) -> list:
        """Arithmetic of each pass of a tensor-core plan (PREC_* values)."""
        out = []
        for i in range(self.info()["sweeps"]):
            v = ctypes.c_int()
            _check(lib().qsim_plan_tc_precision(self.handle, i, ctypes.byref(v)))
            out.append(v.value)
        return out

    def set_tc_precisions(self, prec):
        arr = _arr(prec, np.int32)
        _check(lib().qsim_plan_tc_set_precision(self.handle, len(arr), _p(arr)))

    def info(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().qsim_plan_info(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"sweeps": a.value, "gates": b.value, "mode": c.value}

    def flops(self) -> dict:
        """Flops per amplitude: executed by the staged plan's ops, and of the
        circuit's gates one sweep each."""
        e, c = ctypes.c_double(), ctypes.c_double()
        _check(lib().qsim_plan_flops(self.handle, ctypes.byref(e), ctypes.byref(c)))
        return {"executed": e.value, "circuit": c.value}

    def stage_dump(self, i: int) -> str:
        """Stage i of a staged plan as text (op list, phases, coefficients)."""
        need = ctypes.c_size_t()
        _check(lib().qsim_plan_stage_dump(self.handle, i, None, 0, ctypes.byref(need)))
        buf = ctypes.create_string_buffer(need.value)
        _check(lib().qsim_plan_stage_dump(self.handle, i, buf, need.value, None))
        return buf.value.decode()

    def source(self, dtype: str = "c64") -> str:
        """CUDA source of the plan's specialised stage kernels (staged plans)."""
        need = ctypes.c_size_t()
        dt = C64 if dtype == "c64" else C128
        _check(lib().qsim_plan_source(self.handle, dt, None, 0, ctypes.byref(need)))
        buf = ctypes.create_string_buffer(need.value)
        _check(lib().qsim_plan_source(self.handle, dt, buf, need.value, None))
        return buf.value.decode()

    def describe(self) -> str:
        buf = ctypes.create_string_buffer(1 << 20)
        _check(lib().qsim_plan_describe(self.handle, buf, len(buf)))
        return buf.value.decode()

    def block(self, i: int):
        k = ctypes.c_int()
        t = np.zeros(8, dtype=np.int32)
        _check(lib().qsim_plan_block(self.handle, i, ctypes.byref(k), _p(t), None))
        m = np.zeros((1 << k.value) ** 2 * 2, dtype=np.float64)
        _check(lib().qsim_plan_block(self.handle, i, ctypes.byref(k), _p(t), _p(m)))
        d = 1 << k.value
        return tuple(int(v) for v in t[: k.value]), m.view(np.complex128).reshape(d, d)

    def stages(self) -> list:
        """The stages of a staged plan: dicts with `plain`, `gates` (indices of
        the circuit's gates, in the order applied) and `slots` (tile qubits
        beyond the lanes 0..4)."""
        out = []
        ng = self.info()["gates"]
        for i in range(self.info()["sweeps"]):
            plain, k, ns = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
            g, sl = np.zeros(max(ng, 1), dtype=np.int32), np.zeros(64, dtype=np.int32)
            _check(lib().qsim_plan_stage(self.handle, i, ctypes.byref(plain), ctypes.byref(k), _p(g),
                                         ctypes.byref(ns), _p(sl)))
            out.append({"plain": bool(plain.value), "gates": [int(v) for v in g[: k.value]],
                        "slots": [int(v) for v in sl[: ns.value]]})
        return out

    def tc_passes(self) -> list:
        """The passes of a tensor-core plan as gates on the circuit's qubits:
        dicts with `plain`, `targets`, `controls`, `matrix` and, for fused
        blocks, the diagonal `epilogue` gates applied after the block."""
        out = []
        C = 32  # room for QSIM_MAX_CONTROLS + QSIM_MAX_TARGETS entries
        for i in range(self.info()["sweeps"]):
            plain, k, nc, ne = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
            t, c = np.zeros(8, dtype=np.int32), np.zeros(C, dtype=np.int32)
            _check(lib().qsim_plan_tc_pass(self.handle, i, ctypes.byref(plain), ctypes.byref(k), _p(t),
                                           ctypes.byref(nc), _p(c), None, ctypes.byref(ne)))
            d = 1 << k.value
            m = np.zeros(2 * d * d, dtype=np.float64)
            _check(lib().qsim_plan_tc_pass(self.handle, i, None, None, None, None, None, _p(m), None))
            epi = []
            for e in range(ne.value):
                ek, enc = ctypes.c_int(), ctypes.c_int()
                et, ec = np.zeros(C, dtype=np.int32), np.zeros(C, dtype=np.int32)
                _check(lib().qsim_plan_tc_epilogue(self.handle, i, e, ctypes.byref(ek), _p(et), ctypes.byref(enc),
                                                   _p(ec), None))
                dg = np.zeros(2 << ek.value, dtype=np.float64)
                _check(lib().qsim_plan_tc_epilogue(self.handle, i, e, None, None, None, None, _p(dg)))
                epi.append({"targets": tuple(int(v) for v in et[: ek.value]),
                            "controls": tuple(int(v) for v in ec[: enc.value]), "diag": dg.view(np.complex128)})
            out.append({"plain": bool(plain.value), "targets": tuple(int(v) for v in t[: k.value]),
                        "controls": tuple(int(v) for v in c[: nc.value]),
                        "matrix": m.view(np.complex128).reshape(d, d), "epilogue": epi})
        return out


class SlicePlan:
    """A sliced-state plan: SWAP steps and per-slice segment plans (qsim_slice_plan_build)."""

    def __init__(self, circuit, n_global: int, kmax: int = 4, mode: int = FUSE_STAGED, restore: bool = True):
        qc = circuit if isinstance(circuit, QCircuit) else QCircuit(circuit)
        self.n, self.g, self.L = qc.n, n_global, qc.n - n_global
        h = ctypes.c_void_p()
        _check(lib().qsim_slice_plan_build(qc.handle, n_global, kmax, mode, int(restore), ctypes.byref(h)))
        self.handle = h

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.qsim_slice_plan_destroy(self.handle)
            self.handle = None

    def info(self) -> dict:
        v = [ctypes.c_int() for _ in range(5)]
        _check(lib().qsim_slice_plan_info(self.handle, *[ctypes.byref(x) for x in v]))
        return dict(zip(("n_global", "n_local", "steps", "swaps", "variants"), (x.value for x in v)))

    def steps(self) -> list:
        out = []
        for i in range(self.info()["steps"]):
            t, b, l, ng = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
            km = ctypes.c_uint32()
            _check(lib().qsim_slice_plan_step(self.handle, i, ctypes.byref(t), ctypes.byref(b), ctypes.byref(l),
                                              ctypes.byref(km), ctypes.byref(ng)))
            if t.value == SLICE_SWAP:
                out.append({"type": "swap", "global_bit": b.value, "local_pos": l.value})
            else:
                out.append({"type": "segment", "keymask": km.value, "gates": ng.value})
        return out

    def layout(self) -> list:
        pos = np.zeros(self.n, dtype=np.int32)
        _check(lib().qsim_slice_plan_layout(self.handle, _p(pos)))
        return [int(v) for v in pos]

    def segment_gates(self, step: int, slice_index: int) -> list:
        h = ctypes.c_void_p()
        _check(lib().qsim_slice_segment_circuit(self.handle, step, slice_index, ctypes.byref(h)))
        try:
            return circuit_gates(h)
        finally:
            lib().qsim_circuit_destroy(h)

    def apply_segment(self, step: int, slice_index: int, state: "State"):
        _check(lib().qsim_slice_apply_segment(self.handle, step, slice_index, state.handle))

    def run(self, slices: Sequence, dtype: int, location: int, stream=None):
        ptrs = (ctypes.c_void_p * len(slices))(*[t.data_ptr() for t in slices])
        _check(lib().qsim_slice_run(self.handle, dtype, ptrs, location, _stream_ptr(stream)))


def slice_exchange(a, b, n_local: int, local_pos: int, stream=None):
    dt = C64 if str(a.dtype) == "torch.complex64" else C128
    _check(lib().qsim_slice_exchange(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), n_local, dt,
                                     local_pos, _stream_ptr(stream)))


def slice_pack(slice_t, n_local: int, local_pos: int, bit: int, out, stream=None):
    dt = C64 if str(slice_t.dtype) == "torch.complex64" else C128
    _check(lib().qsim_slice_pack(ctypes.c_void_p(slice_t.data_ptr()), n_local, dt, local_pos, bit,
                                 ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))


def slice_unpack(slice_t, n_local: int, local_pos: int, bit: int, src, stream=None):
    dt = C64 if str(slice_t.dtype) == "torch.complex64" else C128
    _check(lib().qsim_slice_unpack(ctypes.c_void_p(slice_t.data_ptr()), n_local, dt, local_pos, bit,
                                   ctypes.c_void_p(src.data_ptr()), _stream_ptr(stream)))


# ------------------------------------------------------------------ state
class State:
    """A 2^n-amplitude state in a torch CUDA tensor, driven through libqsim."""

    def __init__(self, n: int, dtype: str = "c64", tensor=None, stream=None):
        torch = _torch()
        self.n = n
        self.dtype = C64 if dtype in ("c64", "complex64", C64) else C128
        tdt = torch.complex64 if self.dtype == C64 else torch.complex128
        if tensor is None:
            tensor = torch.empty(1 << n, dtype=tdt, device="cuda")
        assert tensor.dtype == tdt and tensor.numel() == 1 << n and tensor.is_contiguous()
        self.tensor = tensor
        self.stream = stream
        h = ctypes.c_void_p()
        _check(lib().qsim_state_create(n, self.dtype, ctypes.c_void_p(tensor.data_ptr()),
                                       _stream_ptr(stream), ctypes.byref(h)))
        self.handle = h

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.qsim_state_destroy(self.handle)
            self.handle = None

    # -- initialisation / transfer
    def init_zero(self):
        _check(lib().qsim_state_init(self.handle, INIT_ZERO, 0, None)); return self

    def init_null(self):
        """Every amplitude 0 (a slice that holds none of the state's weight)."""
        _check(lib().qsim_state_init(self.handle, INIT_NULL, 0, None)); return self

    def init_basis(self, b: int):
        _check(lib().qsim_state_init(self.handle, INIT_BASIS, b, None)); return self

    def from_host(self, amps: np.ndarray):
        a = _arr(amps, np.complex64 if self.dtype == C64 else np.complex128)
        assert a.size == 1 << self.n
        _check(lib().qsim_state_init(self.handle, INIT_HOST, 0, _p(a)))
        self.synchronize()
        return self

    def from_host_async(self, pinned):
        """Start a host->device copy from a pinned torch tensor (kept alive by the caller)."""
        _check(lib().qsim_state_init(self.handle, INIT_HOST, 0, ctypes.c_void_p(pinned.data_ptr())))
        return self

    def to_host(self) -> np.ndarray:
        out = np.empty(1 << self.n, dtype=np.complex64 if self.dtype == C64 else np.complex128)
        _check(lib().qsim_state_copy_to_host(self.handle, _p(out)))
        return out

    def to_host_into(self, pinned):
        _check(lib().qsim_state_copy_to_host(self.handle, ctypes.c_void_p(pinned.data_ptr())))

    def synchronize(self):
        _check(lib().qsim_synchronize(self.handle))

    # -- gates
    def apply_matrix(self, G, targets: Sequence[int], controls: Sequence[int] = ()):
        m = _arr(np.asarray(G, dtype=np.complex128).view(np.float64), np.float64)
        t = _arr(targets, np.int32)
        c = _arr(controls if len(controls) else [0], np.int32)
        _check(lib().qsim_apply_gate(self.handle, _p(m), _p(t), len(targets),
                                     _p(c) if len(controls) else None, len(controls)))

    def apply(self, g: inputs.Gate):
        if g.name == "matrix":
            return self.apply_matrix(g.matrix, g.targets, g.controls)
        t = _arr(g.targets, np.int32)
        c = _arr(g.controls if len(g.controls) else [0], np.int32)
        prm = _arr(list(g.params) + [0.0] * (4 - len(g.params)), np.float64)
        _check(lib().qsim_apply_named(self.handle, GATE_KIND[g.name], _p(t), len(g.targets),
                                      _p(c) if len(g.controls) else None, len(g.controls), _p(prm)))

    def run(self, circuit):
        qc = circuit if isinstance(circuit, QCircuit) else QCircuit(circuit)
        _check(lib().qsim_run(self.handle, qc.handle))
        return qc

    def run_fused(self, plan: Plan):
        _check(lib().qsim_apply_fused(self.handle, plan.handle))

    # -- measurement
    def probabilities(self, qubits: Sequence[int] | None = None, out=None):
        """Host numpy array, or fills the device tensor ``out`` (float64)."""
        q = _arr(qubits if qubits else [0], np.int32)
        m = len(qubits) if qubits else 0
        size = 1 << (m if m else self.n)
        if out is not None:
            assert out.numel() == size and out.dtype == _torch().float64
            _check(lib().qsim_probabilities(self.handle, _p(q) if m else None, m,
                                            ctypes.c_void_p(out.data_ptr()), 1))
            return out
        host = np.zeros(size, dtype=np.float64)
        _check(lib().qsim_probabilities(self.handle, _p(q) if m else None, m, _p(host), 0))
        return host

    def norm2(self) -> float:
        v = ctypes.c_double()
        _check(lib().qsim_norm2(self.handle, ctypes.byref(v)))
        return v.value

    def sample(self, nshots: int, seed: int, counter0: int = 0, out=None):
        if out is not None:
            _check(lib().qsim_sample(self.handle, nshots, seed, counter0, ctypes.c_void_p(out.data_ptr()), 1))
            return out
        host = np.zeros(max(nshots, 1), dtype=np.uint64)
        _check(lib().qsim_sample(self.handle, nshots, seed & (2**64 - 1), counter0 & (2**64 - 1),
                                 _p(host), 0))
        return host[:nshots]

    def collapse(self, qubits: Sequence[int], outcome: int) -> float:
        """Project on `outcome` of `qubits` (qubits[0] = MSB) and renormalise; returns P."""
        q = _arr(qubits, np.int32)
        p = ctypes.c_double()
        _check(lib().qsim_collapse(self.handle, _p(q), len(q), outcome, ctypes.byref(p)))
        return p.value

    def apply_pauli_phase(self, zmask, coeff, theta: float):
        """psi <- exp(-i theta sum_t coeff[t] Z(zmask[t])) psi (one sweep)."""
        zm, c = _arr(zmask, np.uint64), _arr(coeff, np.float64)
        _check(lib().qsim_apply_pauli_phase(self.handle, len(c), _p(zm), _p(c), float(theta)))
        return self

    def expectation(self, ham: inputs.PauliSum) -> float:
        xm, zm, c = _arr(ham.xmask, np.uint64), _arr(ham.zmask, np.uint64), _arr(ham.coeff, np.float64)
        v = ctypes.c_double()
        _check(lib().qsim_expectation_pauli(self.handle, len(c), _p(xm), _p(zm), _p(c), ctypes.byref(v)))
        return v.value


def sample_probs(p_dev, nshots: int, seed: int, counter0: int = 0, stream=None) -> np.ndarray:
    """Sampler on a device float64 tensor of probabilities (host result)."""
    host = np.zeros(max(nshots, 1), dtype=np.uint64)
    _check(lib().qsim_sample_probs(ctypes.c_void_p(p_dev.data_ptr()), p_dev.numel(), nshots,
                                   seed & (2**64 - 1), counter0 & (2**64 - 1), _p(host), 0,
                                   _stream_ptr(stream)))
    return host[:nshots]


# ------------------------------------------------------------------ gradients
def adjoint_grad(circuit, ham: inputs.PauliSum, params: np.ndarray, dtype: str = "c64", stream=None,
                 psi0: "State | None" = None):
    """Gradients (nsets x nparams) and energies (nsets) by the adjoint method,
    from the start state psi0 (a State of the circuit's width and dtype) or
    |0...0> when psi0 is None."""
    qc = circuit if isinstance(circuit, QCircuit) else QCircuit(circuit)
    params = _arr(np.atleast_2d(params), np.float64)
    nsets, npar = params.shape
    grads = np.zeros((nsets, npar), dtype=np.float64)
    en = np.zeros(nsets, dtype=np.float64)
    xm, zm, c = _arr(ham.xmask, np.uint64), _arr(ham.zmask, np.uint64), _arr(ham.coeff, np.float64)
    _check(lib().qsim_adjoint_grad(qc.handle, None if psi0 is None else psi0.handle,
                                   C64 if dtype == "c64" else C128, nsets, _p(params), len(c),
                                   _p(xm), _p(zm), _p(c), _p(grads), _p(en), _stream_ptr(stream)))
    return grads, en


def adjoint_specialize(mode: int) -> int:
    """Stage kernels compiled for the circuit in adjoint_grad: 1 always, -1
    never, 0 from 20 qubits.  Returns the previous mode."""
    prev = ctypes.c_int()
    _check(lib().qsim_adjoint_specialize(int(mode), ctypes.byref(prev)))
    return prev.value


def adjoint_energy(circuit, ham: inputs.PauliSum, dtype: str = "c64"):
    """A torch.autograd.Function computing <H> for a batch of parameter sets
    (tensor nsets x nparams, float64) whose backward returns the adjoint-method
    gradients computed by the library in the same call."""
    torch = _torch()
    qc = circuit if isinstance(circuit, QCircuit) else QCircuit(circuit)

    class _AdjointEnergy(torch.autograd.Function):
        @staticmethod
        def forward(ctx, theta):
            grads, en = adjoint_grad(qc, ham, theta.detach().cpu().numpy(), dtype)
            ctx.save_for_backward(torch.from_numpy(grads).to(theta.device))
            return torch.from_numpy(en).to(theta.device)

        @staticmethod
        def backward(ctx, gout):
            (grads,) = ctx.saved_tensors
            return gout[:, None] * grads

    return _AdjointEnergy.apply


# ------------------------------------------------------------------ batches
class Batch:
    def __init__(self, circuits: Iterable[inputs.Circuit]):
        self.qcs = [c if isinstance(c, QCircuit) else QCircuit(c) for c in circuits]
        arr = (ctypes.c_void_p * len(self.qcs))(*[q.handle.value for q in self.qcs])
        h = ctypes.c_void_p()
        _check(lib().qsim_batch_create(len(self.qcs), arr, ctypes.byref(h)))
        self.handle = h

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.qsim_batch_destroy(self.handle)
            self.handle = None

    def set_config(self, ctas_per_sm: int = 0, tile_qubits: int = 0):
        _check(lib().qsim_batch_set_config(self.handle, ctas_per_sm, tile_qubits))

    def autotune(self, reps: int = 2, stream=None):
        t, c, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(lib().qsim_batch_autotune(self.handle, _stream_ptr(stream), reps, ctypes.byref(t), ctypes.byref(c),
                                         ctypes.byref(ms)))
        return {"tile_qubits": t.value, "ctas_per_sm": c.value, "ms": ms.value}

    def run(self, out, stream=None):
        _check(lib().qsim_batch_run(self.handle, ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out


# ------------------------------------------------------------------ profiling
def profile_enable(on: bool = True):
    _check(lib().qsim_profile_enable(1 if on else 0))


def profile_reset():
    _check(lib().qsim_profile_reset())


def profile_read() -> dict:
    n = ctypes.c_int()
    _check(lib().qsim_profile_count(ctypes.byref(n)))
    out = {}
    for i in range(n.value):
        name = ctypes.c_char_p(); l = ctypes.c_uint64(); ms = ctypes.c_double(); by = ctypes.c_double()
        fl = ctypes.c_double()
        _check(lib().qsim_profile_get(i, ctypes.byref(name), ctypes.byref(l), ctypes.byref(ms),
                                      ctypes.byref(by), ctypes.byref(fl)))
        if l.value:
            out[name.value.decode()] = {"launches": l.value, "ms": ms.value, "bytes": by.value,
                                        "flops": fl.value}
    return out


def spec_stats() -> dict:
    """Specialised stage kernels compiled in this process: seconds in the
    compiler, programs compiled, programs found in the cache."""
    t, n, h = ctypes.c_double(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().qsim_spec_stats(ctypes.byref(t), ctypes.byref(n), ctypes.byref(h)))
    return {"compile_s": t.value, "compiles": n.value, "cache_hits": h.value}


def launch_count() -> int:
    return int(lib().qsim_launch_count())


def version() -> str:
    return lib().qsim_version().decode()
