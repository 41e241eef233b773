"""Helpers for the GPU parity tests: run the library on device buffers and fetch the maps."""
import numpy as np


def to_device(text):
    import torch
    a = np.ascontiguousarray(text, dtype=np.uint8)
    if not a.flags.writeable:              # (torch warns on read-only arrays; copy those)
        a = a.copy()
    return torch.from_numpy(a).to("cuda:0")


def run(lib, prog, d_text, n, c, dfa=False, tuning=None, with_maps=True):
    """(accept, maps [c][k] numpy uint16 or None) through the C ABI."""
    import torch
    k = prog.info["n_dfa_states"] if dfa else prog.info["k"]
    maps = torch.empty((max(c, 1), k), dtype=torch.int16, device="cuda:0") if with_maps else None
    fn = lib.ridfa_recognize_dfa if dfa else lib.ridfa_recognize
    acc = fn(prog, d_text, n, c, tuning=tuning, d_chunk_maps=maps)
    out = None
    if with_maps:
        out = maps.cpu().numpy().view(np.uint16)[:c]
    return acc, out
