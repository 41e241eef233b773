"""Seeded record-line text built directly in device memory with torch (for multi-GiB texts).

Same record layout and field-length distributions as ``texts.c3_text`` (a different random
stream, so the bytes differ from the numpy generator for the same seed).  torch is only the
array library here; nothing of the recognizer is computed.
"""


def c3_text_torch(n, seed, device="cuda:0", block_records=1 << 22):
    """Record lines until at least n bytes, as a uint8 tensor on `device` (whole lines)."""
    import torch

    from .texts import _SEGS, _TS_LENS
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    nseg = len(_SEGS)
    code_row = torch.tensor([c if k == 2 else k for k, c in _SEGS], dtype=torch.uint8, device=device)
    ts = torch.tensor(_TS_LENS, dtype=torch.int32, device=device)
    var = {12: (1, 10), 14: (1, 10), 16: (1, 7), 18: (1, 13), 20: (1, 4), 22: (1, 4), 24: (1, 4),
           26: (1, 4)}
    parts, total = [], 0
    while total < n:
        need = n - total
        nrec = int(min(block_records, max(16, need // 40 + 16)))
        lens = torch.ones((nrec, nseg), dtype=torch.int32, device=device)
        lens[:, :11] = ts
        for j, (lo, hi) in var.items():
            lens[:, j] = torch.randint(lo, hi, (nrec,), generator=g, device=device, dtype=torch.int32)
        code = code_row.repeat(nrec)
        out = torch.repeat_interleave(code, lens.reshape(-1).to(torch.int64))
        m = out.numel()
        dig = torch.randint(48, 58, (m,), generator=g, device=device, dtype=torch.uint8)
        let = torch.randint(97, 123, (m,), generator=g, device=device, dtype=torch.uint8)
        out = torch.where(out == 0, dig, torch.where(out == 1, let, out))
        del dig, let, lens, code
        if total + m > n:
            nl = torch.nonzero(out == 10).flatten()
            idx = int(torch.searchsorted(nl, torch.tensor([need - 1], device=device)).item())
            out = out[: int(nl[idx].item()) + 1]
        parts.append(out)
        total += out.numel()
    res = torch.cat(parts) if len(parts) > 1 else parts[0]
    return res
