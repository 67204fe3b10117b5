"""Convenience wrapper: owns an lbp_code and torch-allocated buffers.

Allocation and argument marshalling only; decoding is the lbp_decode /
lbp_decode_host call of the C library.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import lbp


def words(bits: int) -> int:
    return (bits + 63) // 64


@dataclass
class DeviceResult:
    err: torch.Tensor        # [B][ceil(n/64)] int64 (uint64 bit patterns)
    converged: torch.Tensor  # [B] uint8
    osd: torch.Tensor        # [B] uint8
    iters: torch.Tensor      # [B] int32
    llr: torch.Tensor | None  # [B][n] float32


class Decoder:
    """One loaded code and a workspace that grows to the largest batch seen.

    The workspace is shared by every call on this object, so calls on
    different streams must not overlap on the GPU (use one Decoder per
    stream for that).  A call on a stream other than torch's current one
    records that stream on the workspace: when a larger batch replaces the
    buffer, the caching allocator hands the old block to other work only
    after that stream has finished with it."""

    def __init__(self, h, priors, device: str | int = "cuda"):
        self.h = h
        self.priors = priors
        self.device = torch.device(device)
        with torch.cuda.device(self.device):
            self.code = lbp.lbp_load_code(h.m, h.n, h.row_ptr, h.col_idx, priors)
        self._ws = None

    def params(self, **kw) -> lbp.lbp_params:
        return lbp.lbp_params_default(**kw)

    def _hold(self, stream):
        if stream is None:
            return
        handle = int(getattr(stream, "cuda_stream", stream))
        with torch.cuda.device(self.device):
            if handle == torch.cuda.current_stream().cuda_stream:
                return
            s = stream if isinstance(stream, torch.cuda.Stream) else torch.cuda.ExternalStream(handle)
        self._ws.record_stream(s)

    def workspace(self, params, num_shots: int, host: bool = False, llr: bool = False, stream=None):
        fn = lbp.lbp_host_workspace_size if host else lbp.lbp_workspace_size
        need = fn(self.code, params, num_shots)
        if need == 0:
            raise ValueError("invalid parameters for this code")
        if host and llr:
            need += ((4 * self.h.n * num_shots + 255) // 256) * 256
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need + 256, dtype=torch.uint8, device=self.device)
        self._hold(stream)
        off = (-self._ws.data_ptr()) % 256
        return self._ws[off:off + need]

    def alloc(self, num_shots: int, want_llr: bool = False) -> DeviceResult:
        d = self.device
        return DeviceResult(
            torch.empty((num_shots, words(self.h.n)), dtype=torch.int64, device=d),
            torch.empty(num_shots, dtype=torch.uint8, device=d),
            torch.empty(num_shots, dtype=torch.uint8, device=d),
            torch.empty(num_shots, dtype=torch.int32, device=d),
            torch.empty((num_shots, self.h.n), dtype=torch.float32, device=d) if want_llr else None)

    def decode(self, syndromes: torch.Tensor, params, want_llr: bool = False,
               out: DeviceResult | None = None, stream=None) -> DeviceResult:
        B = syndromes.shape[0]
        if out is None:
            out = self.alloc(B, want_llr)
        ws = self.workspace(params, B, stream=stream)
        lbp.lbp_decode(self.code, params, B, syndromes, out.err, out.converged, out.osd, out.iters,
                       out.llr, ws, stream)
        return out

    def tune(self, syndromes: torch.Tensor, params, stream=None) -> DeviceResult:
        """lbp_tune on this batch; returns its (valid) decode results."""
        B = syndromes.shape[0]
        out = self.alloc(B)
        lbp.lbp_tune(self.code, params, B, syndromes, out.err, out.converged, out.osd, out.iters,
                     self.workspace(params, B, stream=stream), stream)
        return out

    def decode_host(self, syndromes, params, out: dict, stream=None):
        """syndromes and every array in `out` are pinned CPU tensors."""
        B = syndromes.shape[0]
        ws = self.workspace(params, B, host=True, llr=out.get("llr") is not None, stream=stream)
        lbp.lbp_decode_host(self.code, params, B, syndromes, out["err"], out["converged"],
                            out.get("osd"), out["iters"], out.get("llr"), ws, stream)
        return out

    def close(self):
        self.code.close()
