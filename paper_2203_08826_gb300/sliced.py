"""Sliced states: the multi-GPU scheme of Sec. 3.1 (its figure).

An n-qubit state is split by its top g qubits into 2^g slices of L = n - g
qubits (``qsim_slice_plan_build`` in ``include/qsim.h`` says how gates on the
top qubits are handled).  Three ways to hold the slices:

* ``SlicedState(location="device")`` -- every slice in device memory of this
  process; exchanges are kernels (``qsim_slice_run``).
* ``SlicedState(location="host")`` -- the paper's scheme: the full state in
  page-locked host memory, slices streamed through the GPU in groups.
* ``run_distributed`` -- slices spread over ranks (rank r holds the block of
  slices whose top log2(world) global bits equal r).  An exchange on a global
  bit that selects the rank sends half of every slice to the partner rank
  (point-to-point ``torch.distributed`` send/recv, NCCL on GPUs); every other
  step runs locally through an engine.

The driver logic here only moves buffers and calls the engine; every update
of amplitudes happens in libqsim kernels (``CudaSliceEngine``).
"""
from __future__ import annotations

import math

import numpy as np

from . import binding as _b


def _torch():
    import torch
    return torch


class SlicedState:
    """2^g slices of 2^L amplitudes each, in device or page-locked host memory."""

    def __init__(self, n: int, n_global: int, dtype: str = "c64", location: str = "device"):
        torch = _torch()
        if not 0 <= n_global < n:
            raise ValueError("need 0 <= n_global < n")
        self.n, self.g, self.L = n, n_global, n - n_global
        self.dtype = _b.C64 if dtype in ("c64", _b.C64) else _b.C128
        self.location = {"device": _b.SLICES_DEVICE, "host": _b.SLICES_HOST}[location]
        tdt = torch.complex64 if self.dtype == _b.C64 else torch.complex128
        if self.location == _b.SLICES_DEVICE:
            self.slices = [torch.empty(1 << self.L, dtype=tdt, device="cuda") for _ in range(1 << self.g)]
        else:
            self.slices = [torch.empty(1 << self.L, dtype=tdt, pin_memory=True) for _ in range(1 << self.g)]

    def init_zero(self):
        """|0...0>: slice 0 starts at its first amplitude, every other slice is 0.
        Device slices are written by the library's init kernel (on the current
        stream, which the plan's run uses too); page-locked host slices are
        filled on the host."""
        if self.location == _b.SLICES_DEVICE:
            kind = "c64" if self.dtype == _b.C64 else "c128"
            for i, t in enumerate(self.slices):
                st = _b.State(self.L, kind, tensor=t)
                if i == 0:
                    st.init_zero()
                else:
                    st.init_null()
        else:
            for t in self.slices:
                t.zero_()
            self.slices[0][0] = 1.0
        return self

    def from_host(self, amps: np.ndarray):
        torch = _torch()
        a = np.asarray(amps).astype(_np_dtype(self.dtype)).reshape(1 << self.g, 1 << self.L)
        for i, t in enumerate(self.slices):
            t.copy_(torch.from_numpy(np.ascontiguousarray(a[i])))
        return self

    def to_host(self) -> np.ndarray:
        _torch().cuda.synchronize()
        return np.concatenate([t.cpu().numpy() for t in self.slices])

    def run(self, plan: "_b.SlicePlan", stream=None):
        if plan.g != self.g or plan.L != self.L:
            raise ValueError("plan and state are sliced differently")
        plan.run(self.slices, self.dtype, self.location, stream)
        return self


def _np_dtype(dt):
    return np.complex64 if dt == _b.C64 else np.complex128


# ------------------------------------------------------------------ several ranks
class CudaSliceEngine:
    """Slice updates through libqsim on CUDA tensors of this rank's device."""

    def __init__(self, plan: "_b.SlicePlan"):
        self.plan = plan
        self._states = {}

    def apply_segment(self, step: int, index: int, buf):
        st = self._states.get(buf.data_ptr())
        if st is None:
            st = _b.State(self.plan.L, "c64" if str(buf.dtype) == "torch.complex64" else "c128", tensor=buf)
            self._states[buf.data_ptr()] = st
        self.plan.apply_segment(step, index, st)

    def exchange(self, a, b, local_pos: int):
        _b.slice_exchange(a, b, self.plan.L, local_pos)

    def pack(self, buf, local_pos: int, bit: int):
        out = _torch().empty(buf.numel() // 2, dtype=buf.dtype, device=buf.device)
        _b.slice_pack(buf, self.plan.L, local_pos, bit, out)
        return out

    def unpack(self, buf, local_pos: int, bit: int, src):
        _b.slice_unpack(buf, self.plan.L, local_pos, bit, src)

    def synchronize(self):
        _torch().cuda.current_stream().synchronize()


def owned_slices(g: int, rank: int, world: int) -> range:
    """The slices rank `rank` of `world` holds (world a power of two <= 2^g)."""
    if world & (world - 1) or world > (1 << g):
        raise ValueError("world size must be a power of two no larger than the number of slices")
    per = (1 << g) // world
    return range(rank * per, (rank + 1) * per)


def run_distributed(plan: "_b.SlicePlan", slices: dict, engine, group=None):
    """Run every step of `plan` on this rank's slices ({slice index: buffer}).

    Exchanges between slices of one rank go to ``engine.exchange``; an
    exchange on a rank-selecting global bit packs, per slice, the half whose
    local bit differs from the slice's global bit, swaps it with the partner
    rank (send and receive posted together, slices in increasing order on
    both sides, so the pairs line up) and unpacks what arrived into the same
    half.  The slices are pipelined two deep: slice i is packed and its
    transfer posted before the host waits for slice i - 1's transfer, whose
    half is unpacked while slice i's is in flight (two send and two receive
    buffers at a time).
    """
    torch = _torch()
    import torch.distributed as dist
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    g = plan.g
    own = owned_slices(g, rank, world)
    if sorted(slices) != list(own):
        raise ValueError(f"rank {rank} must hold slices {own.start}..{own.stop - 1}")
    rank_bits = int(math.log2(world))
    local_bits = g - rank_bits  # global bits below these select a slice within the rank
    for k, st in enumerate(plan.steps()):
        if st["type"] == "segment":
            for i in own:
                engine.apply_segment(k, i, slices[i])
            continue
        b, l = st["global_bit"], st["local_pos"]
        if b < local_bits:
            for i in own:
                if not (i >> b) & 1:
                    engine.exchange(slices[i], slices[i | (1 << b)], l)
            continue
        peer_bit = b - local_bits
        peer = rank ^ (1 << peer_bit)
        if group is not None:
            peer = dist.get_global_rank(group, peer)
        mybit = (rank >> peer_bit) & 1
        half_bit = 1 - mybit  # the half this rank gives away and receives
        pending = None  # (slice, send, recv, requests) of the transfer in flight
        for i in own:
            send = engine.pack(slices[i], l, half_bit)
            recv = torch.empty_like(send)
            engine.synchronize()
            ops = [dist.P2POp(dist.isend, torch.view_as_real(send), peer, group),
                   dist.P2POp(dist.irecv, torch.view_as_real(recv), peer, group)]
            reqs = dist.batch_isend_irecv(ops)
            if pending is not None:
                _finish_transfer(engine, slices, l, half_bit, pending)
            pending = (i, send, recv, reqs)
        if pending is not None:
            _finish_transfer(engine, slices, l, half_bit, pending)
    engine.synchronize()


def _finish_transfer(engine, slices, l, half_bit, pending):
    i, _send, recv, reqs = pending  # the send buffer lives until its request is done
    for req in reqs:
        req.wait()
    engine.unpack(slices[i], l, half_bit, recv)
