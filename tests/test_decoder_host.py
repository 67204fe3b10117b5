"""Host logic of the Decoder wrapper that needs no GPU: which streams are
recorded on the shared workspace (torch's CUDA calls are replaced by fakes)."""
import contextlib

import torch

from paper_2605_00038_gb300.decoder import Decoder


class _Buf:
    def __init__(self):
        self.recorded = []

    def record_stream(self, s):
        self.recorded.append(s)


class _Stream:
    def __init__(self, handle):
        self.cuda_stream = handle


def test_workspace_records_only_streams_other_than_the_current_one(monkeypatch):
    monkeypatch.setattr(torch.cuda, "device", lambda d: contextlib.nullcontext())
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a: _Stream(7))
    monkeypatch.setattr(torch.cuda, "ExternalStream", lambda h: ("external", h))
    dec = Decoder.__new__(Decoder)
    dec.device = torch.device("cuda")
    dec._ws = _Buf()
    dec._hold(None)                  # torch's current stream, implicitly
    dec._hold(_Stream(7))            # the current stream, explicitly
    dec._hold(7)                     # its raw handle
    assert dec._ws.recorded == []
    dec._hold(9)                     # a raw handle of another stream
    dec._hold(_Stream(11))           # a stream object that is not torch.cuda.Stream
    assert dec._ws.recorded == [("external", 9), ("external", 11)]
