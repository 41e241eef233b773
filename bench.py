#!/usr/bin/env python
"""Throughput of the GB300 RID recognizer on one text resident in HBM.

One step = one pass of the whole hot path over the workload: ridfa_recognize_async (reach
kernel over every chunk and interface slot, then the join kernel that yields the accept bit).
Default workload: the 4 GiB ASCII record-line text against (TS,ID,FLOAT,WORD,IP\\n)*, cut into
2^17 chunks.  The text (4 GiB) is larger than L2, so no flush is needed between steps.

Printed (rank 0, one JSON line): value = input GB/s (device-timed, CUDA events on the launch
stream), the all-states DFA comparator on the same text, the reach kernel's roofline against
the measured HBM copy bandwidth, SM clocks sampled during the timed region, an end-to-end
figure through the C ABI with the text copied from pinned host memory every step, and the
oracle (Thompson state-set simulation, one host core) on a bounded sample as the CPU baseline.

--impl reference times the oracle on the host cores instead (the comparison arm).
With torchrun (N > 1) every rank recognises its own replica of the workload (weak scaling);
there is no data-path collective.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "input GB/s on 1 GB300 (RI-DFA vs all-states DFA), batched GB/s, served p99 ms"

WORKLOADS = {
    # name: (description, default bytes, default chunks)
    "c3": ("ASCII record lines (TS,ID,FLOAT,WORD,IP\\n)*, literal field order", 4 << 30, 1 << 17),
    "c3any": ("ASCII record lines, any field per column ((F)(,F)*\\n)*", 4 << 30, 1 << 17),
    "c2": ("DNA motif RE with the {2,4} codon repeat, i.i.d. ACGT", 1 << 30, 1 << 16),
    "c1": ("((A|C)*G(T|A)+C)*, walk on the minimal DFA", 1 << 20, 64),
    "regexp": ("(a|b)*a(a|b){k}, i.i.d. a/b (the paper's regexp family)", 1 << 30, 1 << 17),
}


REGEXP_K = 7   # (a|b)*a(a|b){7}: the minimal DFA has 256 states (the comparator's limit), k = 9


def workload_re(name, k=REGEXP_K):
    import textgen
    return {"c3": textgen.C3_RE, "c3any": textgen.C3_RE_ANYFIELD,
            "c2": textgen.C2_RE.replace("{20,60}", "{2,4}"), "c1": textgen.C1_RE,
            "regexp": textgen.regexp_family_re(k)}[name]


def make_text(name, n, seed, device):
    import torch

    import textgen
    if name in ("c3", "c3any"):
        return textgen.c3_text_torch(n, seed, device=device)
    if name in ("c2", "regexp"):
        g = torch.Generator(device=device)
        g.manual_seed(seed)
        alpha = b"ACGT" if name == "c2" else b"ab"
        lut = torch.tensor(list(alpha), dtype=torch.uint8, device=device)
        return lut[torch.randint(0, len(alpha), (n,), generator=g, device=device)]
    x = textgen.c1_text(n, seed)
    return torch.from_numpy(x).to(device)


def sample_text_numpy(name, n, seed):
    import numpy as np

    import textgen
    if name in ("c3", "c3any"):
        return textgen.c3_text(n, seed)
    if name == "c2":
        return textgen.c2_text(n, seed)
    if name == "regexp":
        return textgen.regexp_family_text(n, seed)
    return textgen.c1_text(n, seed)


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, max clock, throttle reasons)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=self.file, stderr=subprocess.DEVNULL)
            # start timing only once the sampler is producing samples
            t0 = time.time()
            while time.time() - t0 < 5.0 and self.proc.poll() is None:
                if os.path.getsize(self.file.name) > 0:
                    break
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None:
            return None
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.file.name)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, flags in rows for i, fl in enumerate(flags)
                          if fl.lower() in ("active", "1", "yes")})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons, "samples": len(rows)}


# DRAM bytes (read + write) per text byte of the reach kernel, from one ncu capture of it
# (record-line RE, 1 GiB, 155,648 chunks: dram__bytes_read.sum + dram__bytes_write.sum); applied
# to the record-line workload in the same launch shape (Rep16 tables, cooperative staging), scaled
# by the text bytes.  Must be re-measured (or dropped) whenever that kernel changes.
REACH_TRAFFIC = {"workload": "c3", "kernel": "rid_reach_kernel<4, LutRep<true>, 1024, 2>",
                 "dram_bytes_per_text_byte": 1.0312}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def cpu_baseline(name, re_src, budget_s=12.0, seed=7):
    """The oracle (Thompson state-set simulation, one core) on a bounded sample of the workload."""
    from oracle.recognizer import SerialRecognizer
    ser = SerialRecognizer(re_src)
    n = 4 << 20
    x = sample_text_numpy(name, n, seed)
    t = time.perf_counter()
    ser.accepts(x)
    dt = time.perf_counter() - t
    rate = x.size / max(dt, 1e-9)
    n2 = int(min(2 << 30, max(n, rate * budget_s)))
    if n2 > x.size:
        x = sample_text_numpy(name, n2, seed + 1)
        t = time.perf_counter()
        ser.accepts(x)
        dt = time.perf_counter() - t
    return {"value": round(x.size / dt / 1e9, 6), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"{x.size} bytes of the same workload's text generator, one Thompson "
                      f"state-set simulation pass ({dt:.1f} s)"}


def measure_cpu_context(lib, prog, hx, acc, has_dfa, serial_cap=1 << 30):
    """The recognition on the host's cores (ridfa_cpu_recognize): the serial table loop on a
    prefix of at most serial_cap bytes, and one chunk per hardware thread over the whole text,
    RID and all-states DFA; GB/s of one timed pass each."""
    threads = os.cpu_count() or 1
    pre = hx[:min(hx.size, serial_cap)]
    out = {"unit": "GB/s", "threads": threads, "serial_sample_bytes": int(pre.size),
           "chunked_bytes": int(hx.size), "chunks": threads}

    def rate(x, c, t, dfa):
        t0 = time.perf_counter()
        a = lib.ridfa_cpu_recognize(prog, x, c, dfa=dfa, n_threads=t)
        return a, round(x.size / (time.perf_counter() - t0) / 1e9, 3)

    _, out["serial_rid"] = rate(pre, 1, 1, False)
    a, out["chunked_rid"] = rate(hx, threads, threads, False)
    assert a == acc, "host and device recognition disagree"
    if has_dfa:
        _, out["serial_dfa"] = rate(pre, 1, 1, True)
        a, out["chunked_dfa"] = rate(hx, threads, threads, True)
        assert a == acc, "host all-states DFA and device recognition disagree"
    return out


def run_reference_multi(args, name):
    """The oracle on the batched or served workload: a bounded sample of its texts, item by item.
    (The workload's random REs are selected with the library's host compiler; the timed path is
    the oracle alone.)"""
    import numpy as np

    import paper_2412_14975_gb300 as lib
    from oracle.recognizer import SerialRecognizer
    if name == "batch":
        res, texts = build_batch_workload_host(lib, 64, args.seed)
        rid = [i % len(res) for i in range(len(texts))]
    else:
        res, _, texts, rid = build_served_workload(lib, 32, 128, args.seed)
    sers = {}
    order = list(range(len(texts)))
    for i in range(args.warmup):
        j = order[i % len(order)]
        sers.setdefault(rid[j], SerialRecognizer(res[rid[j]])).accepts(texts[j])
    per_step = 4 << 20
    svc = []
    t = time.perf_counter()
    nbytes = 0
    pos = 0
    for _ in range(args.steps):
        got = 0
        while got < per_step:
            j = order[pos % len(order)]
            pos += 1
            t1 = time.perf_counter()
            sers.setdefault(rid[j], SerialRecognizer(res[rid[j]])).accepts(texts[j])
            svc.append((time.perf_counter() - t1) * 1e3)
            got += texts[j].size
        nbytes += got
    dt = time.perf_counter() - t
    v = nbytes / dt / 1e9
    line = {"metric": METRIC, "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic", "impl": "reference",
            "value": round(v, 6),
            "config": {"workload": f"{name}: oracle over {per_step} bytes of the workload's texts per step",
                       "texts_in_sample": len(texts)},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "value": round(v, 6), "unit": "GB/s",
                             "sample": f"{per_step} bytes per step, item by item"},
            "e2e": {"value": round(v, 6), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if name == "served":
        # one request at a time: its service time bounds the latency from below (the oracle cannot
        # keep up with the offered rates, so its queueing latency grows without bound)
        line["value"] = round(float(np.percentile(svc, 99)), 3)
        line["unit"] = "ms"
        line["higher_is_better"] = False
        line["config"]["note"] = "value = p99 of per-request service time (unloaded); GB/s in cpu_baseline"
    print(json.dumps(line), flush=True)


def run_reference(args, rank):
    if rank != 0:
        return
    name = args.workload
    if name in ("batch", "served"):
        run_reference_multi(args, name)
        return
    re_src = workload_re(name, args.k)
    from oracle.recognizer import SerialRecognizer
    ser = SerialRecognizer(re_src)
    per_step = 16 << 20
    samples = [sample_text_numpy(name, per_step, 1000 + i) for i in range(2)]
    for i in range(args.warmup):
        ser.accepts(samples[i % 2])
    t = time.perf_counter()
    nbytes = 0
    for i in range(args.steps):
        x = samples[i % 2]
        ser.accepts(x)
        nbytes += x.size
    dt = time.perf_counter() - t
    v = nbytes / dt / 1e9
    desc, _, _ = WORKLOADS[name]
    line = {"metric": METRIC, "value": round(v, 6), "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": f"{name}: {desc}", "sample_bytes_per_step": per_step},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "value": round(v, 6), "unit": "GB/s",
                             "sample": f"{per_step} bytes per step of the workload's text generator"},
            "e2e": {"value": round(v, 6), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def select_batch_res(lib, seed):
    """The batched configuration's 16 REs: the 3 single-text REs and the first 13 random (R)* REs
    whose RI-DFA has 10..5000 states and at most 256 interface slots."""
    import textgen.batch as tb
    res = tb.standard_res()
    kept = []
    for r, body, alpha in tb.random_re_candidates(seed, 400):
        try:
            p = lib.ridfa_compile(r, build_dfa=False)
        except lib.RidfaError:
            continue
        if 10 <= p.info["n_states"] <= 5000 and p.info["k"] <= lib.RIDFA_MAX_SLOTS:
            kept.append((r, body, alpha))
        if len(kept) == 13:
            break
    return res + kept


def build_batch_workload_host(lib, n_texts, seed):
    """Host side of the batched configuration: (REs, texts); text j uses RE j mod 16."""
    import textgen.batch as tb
    res = select_batch_res(lib, seed)
    texts = [x for _, _, x, _ in tb.batch_texts(res, n_texts, seed + 1)]
    return [r for r, _, _ in res], texts


def build_batch_workload(lib, torch, dev, n_texts, seed):
    """The batched configuration: n_texts texts (lognormal lengths) over 16 REs, resident in one
    16-byte-aligned device buffer.  Returns (progs, items, total_bytes, device buffer, REs, texts)."""
    import numpy as np

    import textgen.batch as tb
    res = select_batch_res(lib, seed)
    progs = [lib.ridfa_compile(r, build_dfa=False) for r, _, _ in res]
    texts, rid = [], []
    for j, r, x, _ in tb.batch_texts(res, n_texts, seed + 1):
        texts.append(x)
        rid.append(r)
    offs = np.zeros(len(texts), dtype=np.int64)
    pos = 0
    for i, x in enumerate(texts):
        offs[i] = pos
        pos = (pos + x.size + 15) & ~15
    host = torch.empty(pos, dtype=torch.uint8, pin_memory=True)
    hv = host.numpy()
    for o, x in zip(offs, texts):
        hv[o:o + x.size] = x
    d = host.to(dev)
    base = d.data_ptr()
    items = [(base + int(o), int(x.size), r, 0) for o, x, r in zip(offs, texts, rid)]
    total = int(sum(x.size for x in texts))
    return progs, items, total, d, [r for r, _, _ in res], texts


def oracle_accepts(res, texts, rid, idx):
    """Accept bits of texts[i] for i in idx by the oracle (Thompson state-set simulation)."""
    from oracle.recognizer import SerialRecognizer
    sers = {}
    out = {}
    for i in idx:
        r = rid[i]
        if r not in sers:
            sers[r] = SerialRecognizer(res[r])
        out[int(i)] = bool(sers[r].accepts(texts[i]))
    return out


def measure_batch(args, lib, torch, dev, stream, world, rank, steps, warmup, oracle_sample=256):
    """The batched configuration: one CUDA graph over every (text, RE) item, replayed `steps`
    times; the plain one-text-per-launch path on the same items; accept bits of a seeded sample
    of items against the oracle."""
    import numpy as np
    t0 = time.perf_counter()
    progs, items, total, d, res, texts = build_batch_workload(lib, torch, dev, args.batch_texts, args.seed)
    gen_s = time.perf_counter() - t0
    acc = torch.zeros(len(items), dtype=torch.uint8, device=dev)
    t0 = time.perf_counter()
    b = lib.ridfa_batch_create(progs, items, acc, chunk_len=args.batch_chunk_len,
                               block_warps=args.batch_warps, set_mode=args.batch_set_mode)
    create_s = time.perf_counter() - t0
    st = lib.ridfa_batch_get_stats(b)
    for _ in range(warmup):
        lib.ridfa_batch_run(b, stream=stream)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            lib.ridfa_batch_run(b, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * total * steps / (ms / 1e3) / 1e9
    got = acc.cpu().numpy().astype(bool)
    b.close()
    # the plain one-text-per-launch path on the same texts (same chunk length), for comparison
    L = st["chunk_len"]
    acc1 = torch.zeros(1, dtype=torch.uint8, device=dev)

    def one_pass():
        for (ptr, n, r, _) in items:
            lib.ridfa_recognize_async(progs[r], ptr, n, max(1, min(n, (n + L - 1) // L)), acc1, stream=stream)
    single_value = None
    if not args.no_batch_single:
        one_pass()
        torch.cuda.synchronize()
        e0.record(stream)
        one_pass()
        e1.record(stream)
        torch.cuda.synchronize()
        single_value = total / (e0.elapsed_time(e1) / 1e3) / 1e9
    # each RE's texts end to end as one long text (every RE here is star-closed, so the
    # concatenation of its members is a member), recognized alone at the best of the batch's chunk
    # length and three large chunk counts: the rate each RE reaches by itself; the batch against
    # the sum of those times shows what mixing programs in one graph costs or gains
    per_re = []
    sep_ms = 0.0
    if not args.no_batch_per_re:
        rid_all = [it[2] for it in items]
        for r in range(len(progs)):
            xs = [texts[i] for i in range(len(texts)) if rid_all[i] == r and texts[i].size]
            if not xs:
                continue
            cat = np.concatenate(xs)
            dt = torch.from_numpy(cat).to(dev)
            best = None
            for c in sorted({max(1, min(cat.size, (cat.size + L - 1) // L)), 65536, 131072, 155648}):
                if c > cat.size:
                    continue
                lib.ridfa_recognize_async(progs[r], dt.data_ptr(), cat.size, c, acc1, stream=stream)
                torch.cuda.synchronize()
                e0.record(stream)
                for _ in range(3):
                    lib.ridfa_recognize_async(progs[r], dt.data_ptr(), cat.size, c, acc1, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                t = e0.elapsed_time(e1) / 3
                if best is None or t < best[0]:
                    best = (t, c)
            sep_ms += best[0]
            per_re.append({"re": r, "bytes": int(cat.size), "chunks": int(best[1]),
                           "GBps": round(cat.size / (best[0] / 1e3) / 1e9, 1)})
            del dt
        torch.cuda.empty_cache()
    # accept bits of a seeded sample of items against the oracle
    rid = [it[2] for it in items]
    rng = np.random.Generator(np.random.PCG64(5))
    sample = rng.choice(len(items), size=min(oracle_sample, len(items)), replace=False)
    t0 = time.perf_counter()
    want = oracle_accepts(res, texts, rid, sample)
    oracle_s = time.perf_counter() - t0
    mism = sum(int(want[int(i)] != bool(got[i])) for i in sample)
    sample_bytes = int(sum(texts[int(i)].size for i in sample))
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = {"value": round(sample_bytes / oracle_s / 1e9, 6), "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"{len(sample)} sampled batch items ({sample_bytes} bytes), Thompson state-set simulation"}
    return {"value": round(value, 3), "unit": "GB/s", "steps": steps, "warmup": warmup,
            "ms_per_step": round(ms / steps, 4),
            "single_text_per_launch_GBps": round(single_value, 3) if single_value else None,
            "batched_over_single": round(value / single_value, 3) if single_value else None,
            "per_re_alone": per_re or None,
            "per_re_alone_GBps": round(total / (sep_ms / 1e3) / 1e9, 3) if sep_ms else None,
            "batched_over_per_re_alone": round(value / (total / (sep_ms / 1e3) / 1e9), 3) if sep_ms else None,
            "config": {"workload": f"batched: {len(items)} texts, lognormal median 256 KiB sigma 1, "
                                   f"16 REs (3 single-text + 13 random), half mutated, one CUDA graph",
                       "total_bytes": total, "chunk_len": L, "block_warps": st["block_warps"],
                       "set_mode": st["set_mode"], "chunks": st["total_chunks"],
                       "launches_in_graph": st["n_launches"], "tasks": st["n_tasks"],
                       "join_segments": st["n_segments"], "graph": bool(st["graph"]),
                       "accepted": int(got.sum()), "generate_s": round(gen_s, 1),
                       "create_s": round(create_s, 2), "l2": "inputs larger than L2, no flush"},
            "oracle_check": {"items": len(sample), "bytes": sample_bytes, "mismatches": mism,
                             "accepted": int(sum(want.values()))},
            "clocks": clk.summary(), "cpu_baseline": cpu,
            "gpu_launches": steps * st["n_launches"]}


def run_batch(args, lib, torch, dev, stream, world, rank):
    r = measure_batch(args, lib, torch, dev, stream, world, rank, args.steps, args.warmup)
    if rank == 0:
        line = {"metric": METRIC, "value": r["value"], "unit": "GB/s", "n_gpus": world,
                "steps": r["steps"], "warmup": r["warmup"], "ms_per_step": r["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
                "data": "synthetic", "config": r["config"],
                "single_text_per_launch_GBps": r["single_text_per_launch_GBps"],
                "batched_over_single": r["batched_over_single"], "oracle_check": r["oracle_check"],
                "per_re_alone": r["per_re_alone"], "per_re_alone_GBps": r["per_re_alone_GBps"],
                "batched_over_per_re_alone": r["batched_over_per_re_alone"],
                "clocks": r["clocks"], "cpu_baseline": r["cpu_baseline"], "gpu_launches": r["gpu_launches"]}
        print(json.dumps(line), flush=True)


def build_served_workload(lib, n_res, n_pool, seed):
    """The served configuration: n_res resident REs (the 3 single-text REs + random ones) and a pool
    of host texts (lognormal lengths, median 64 KiB, sigma 1, at most 16 MiB) that requests draw
    from.  Returns (REs, programs, texts, RE index of each text)."""
    import numpy as np

    import textgen.batch as tb
    res = tb.standard_res()
    for r, body, alpha in tb.random_re_candidates(seed, 2000):
        if len(res) == n_res:
            break
        try:
            p = lib.ridfa_compile(r, build_dfa=False)
        except lib.RidfaError:
            continue
        if 10 <= p.info["n_states"] <= 5000 and p.info["k"] <= lib.RIDFA_MAX_SLOTS:
            res.append((r, body, alpha))
    progs = [lib.ridfa_compile(r, build_dfa=False) for r, _, _ in res]
    texts, rid = [], []
    for _, r, x, _ in tb.batch_texts(res, n_pool, seed + 1, median=64 << 10, sigma=1.0):
        texts.append(np.ascontiguousarray(x[: 16 << 20]))
        rid.append(r)
    return [r for r, _, _ in res], progs, texts, rid


def measure_served(args, lib, torch, dev, rank, rates, seconds):
    """Open-loop Poisson load on the server at each rate, driven by the library's C load
    generator (ridfa_bench_served_poisson, so the client's cost is not Python's): latency =
    result posted - scheduled arrival.  Every request's accept bit is checked against the
    oracle's answer for its text; the one-text-per-launch path on the same mix is timed beside."""
    import numpy as np
    t0 = time.perf_counter()
    res, progs, texts, rid = build_served_workload(lib, 32, args.served_pool, args.seed)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    want_map = oracle_accepts(res, texts, rid, range(len(texts)))
    want = np.array([want_map[i] for i in range(len(texts))])
    oracle_s = time.perf_counter() - t0
    srv = lib.Server(n_streams=3, arena_bytes=4 << 30, max_batch_requests=8192, max_batch_bytes=512 << 20,
                     chunk_len=args.batch_chunk_len, device_budget=args.served_budget)
    slots = [srv.add_program(p) for p in progs]
    pslots = [slots[r] for r in rid]
    lens = np.array([x.size for x in texts])
    # warm the server (a short run at the lowest rate, unreported)
    srv.bench_poisson(pslots, texts, rates[0], min(1.0, seconds), args.seed + 99)
    results = []
    total_mism = 0

    def one_rate(rate, secs, seed, device_texts=None):
        st0 = srv.stats()
        recs, wall = srv.bench_poisson(pslots, texts, rate, secs, seed, device_texts=device_texts)
        st1 = srv.stats()
        lat = np.sort(recs["latency_us"] / 1e3)
        slat = np.sort(recs["server_us"] / 1e3)
        mism = int(np.count_nonzero((recs["status"] != 0) |
                                    (recs["accept"].astype(bool) != want[recs["text"]])))
        nb = st1["batches"] - st0["batches"]
        hist = [a - b for a, b in zip(st1["batch_hist"], st0["batch_hist"])]
        nbytes = int(lens[recs["text"]].sum())
        return {"offered_rps": rate, "requests": int(len(recs)),
                "achieved_rps": round(len(recs) / wall, 1),
                "GBps": round(nbytes / wall / 1e9, 3),
                "p50_ms": round(float(np.percentile(lat, 50)), 3),
                "p99_ms": round(float(np.percentile(lat, 99)), 3),
                "max_ms": round(float(lat[-1]), 3),
                "server_p50_ms": round(float(np.percentile(slat, 50)), 3),
                "server_p99_ms": round(float(np.percentile(slat, 99)), 3),
                "batches": nb, "mean_batch": round(len(recs) / max(nb, 1), 1),
                "batch_hist_log2": hist[:max([i + 1 for i, h in enumerate(hist) if h] or [1])],
                "busy_retries": int(recs["busy_retries"].sum()),
                "oracle_mismatches": mism}

    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for q, rate in enumerate(rates):
            results.append(one_rate(rate, seconds, args.seed + 7 + q))
            total_mism += results[-1]["oracle_mismatches"]
    # the same mix from device-resident texts (submitted in place: no client copy into the
    # arena), at rates a host-copying client thread cannot offer: the server's own capacity
    dev_results = []
    dev_rates = [int(r) for r in args.served_device_rates.split(",") if r]
    if dev_rates:
        offs = np.zeros(len(texts), dtype=np.int64)
        pos = 0
        for i, x in enumerate(texts):
            offs[i] = pos
            pos = (pos + x.size + 15) & ~15
        hbuf = np.zeros(max(pos, 16), np.uint8)
        for o, x in zip(offs, texts):
            hbuf[o:o + x.size] = x
        dpool = torch.from_numpy(hbuf).to(dev)
        dtexts = [(dpool.data_ptr() + int(o), int(x.size)) for o, x in zip(offs, texts)]
        with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk_dev:
            for q, rate in enumerate(dev_rates):
                dev_results.append(one_rate(rate, args.served_device_seconds, args.seed + 71 + q, dtexts))
                total_mism += dev_results[-1]["oracle_mismatches"]
        del dpool
    stats = srv.stats()
    srv.close()
    # one text per launch on the same request mix: copy, recognise, read the bit, one by one
    # (1 KiB chunks unless given: what the server's adaptive rule picks for a lone request)
    L = args.batch_chunk_len or 1024
    pin = [torch.from_numpy(texts[j]).pin_memory() for j in range(min(len(texts), 512))]
    d_buf = torch.empty(max(int(lens.max()), 16), dtype=torch.uint8, device=dev)
    t0 = time.perf_counter()
    nb1 = 0
    for j, h in enumerate(pin):
        n = h.numel()
        if n == 0:
            continue
        d_buf[:n].copy_(h, non_blocking=True)
        lib.ridfa_recognize(progs[rid[j]], d_buf, n, max(1, min(n, (n + L - 1) // L)))
        nb1 += n
    dt1 = time.perf_counter() - t0
    single = {"requests": len(pin), "GBps": round(nb1 / dt1 / 1e9, 3), "rps": round(len(pin) / dt1, 1)}
    return {"rates": results, "seconds_per_rate": seconds, "single_text_per_launch": single,
            "device_texts": ({"rates": dev_results, "seconds_per_rate": args.served_device_seconds,
                              "clocks": clk_dev.summary()} if dev_results else None),
            "config": {"workload": f"served: Poisson arrivals over {len(res)} resident REs, host texts "
                                   f"lognormal median 64 KiB sigma 1 (max 16 MiB), {seconds} s per rate",
                       "pool_texts": len(texts), "pool_mean_bytes": int(lens.mean()),
                       "generate_s": round(gen_s, 1), "n_streams": 3,
                       "device_budget": args.served_budget or None,
                       "chunk_len": args.batch_chunk_len or "adaptive (1-8 KiB per batch)",
                       "client": "ridfa_bench_served_poisson (C, open loop)"},
            "oracle_check": {"requests": int(sum(r["requests"] for r in results + dev_results)),
                             "mismatches": total_mism,
                             "pool_oracle_s": round(oracle_s, 1)},
            "server_stats": stats, "clocks": clk.summary()}


def run_served(args, lib, torch, dev, rank):
    rates = [int(r) for r in args.served_rates.split(",")]
    r = measure_served(args, lib, torch, dev, rank, rates, args.served_seconds)
    ref = next((x for x in r["rates"] if x["offered_rps"] == args.served_ref_rate), r["rates"][-1])
    if rank == 0:
        cfg = dict(r["config"])
        cfg["workload"] += f"; value = p99 at {ref['offered_rps']} req/s"
        line = {"metric": METRIC, "value": ref["p99_ms"], "unit": "ms", "n_gpus": 1,
                "steps": len(rates), "warmup": args.warmup, "ms_per_step": None,
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
                "data": "synthetic", "config": cfg,
                "rates": r["rates"], "single_text_per_launch": r["single_text_per_launch"],
                "device_texts": r["device_texts"],
                "oracle_check": r["oracle_check"], "server_stats": r["server_stats"], "clocks": r["clocks"],
                "e2e": {"value": ref["GBps"], "unit": "GB/s",
                        "h2d_bytes_per_step": r["config"]["pool_mean_bytes"], "d2h_bytes_per_step": 1},
                "gpu_launches": None}
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS) + ["batch", "served"])
    ap.add_argument("--served-rates", default="2000,5000,10000,20000,50000",
                    help="--workload served: Poisson rates (req/s)")
    ap.add_argument("--served-seconds", type=float, default=60.0,
                    help="--workload served: seconds of arrivals per rate (the configured 60 s)")
    ap.add_argument("--served-ref-rate", type=int, default=10000)
    ap.add_argument("--served-device-rates", default="100000,200000,400000",
                    help="rates also offered from device-resident texts (the server's own capacity); empty to skip")
    ap.add_argument("--served-device-seconds", type=float, default=2.0)
    ap.add_argument("--served-budget", type=int, default=0,
                    help="server device budget in bytes (tables + texts + scratch; 0 = none)")
    ap.add_argument("--no-batched", action="store_true",
                    help="default workload: skip the batched configuration's measurement")
    ap.add_argument("--no-served", action="store_true",
                    help="default workload: skip the served configuration's measurement")
    ap.add_argument("--combined-batch-steps", type=int, default=10)
    ap.add_argument("--combined-served-rates", default="2000,10000,50000")
    ap.add_argument("--combined-served-seconds", type=float, default=10.0)
    ap.add_argument("--served-pool", type=int, default=2048)
    ap.add_argument("--batch-texts", type=int, default=10000)
    ap.add_argument("--batch-chunk-len", type=int, default=0, help="0 = autotune")
    ap.add_argument("--batch-warps", type=int, default=0, help="warps per block of the batch's reach launches (0 = autotune)")
    ap.add_argument("--batch-set-mode", type=int, default=0, help="batch set path: 0 autotune, 1 on, 2 off")
    ap.add_argument("--no-batch-single", action="store_true",
                    help="skip the one-text-per-launch comparison of the batched workload")
    ap.add_argument("--no-batch-per-re", action="store_true",
                    help="skip timing each batch RE alone on the concatenation of its texts")
    ap.add_argument("--text-bytes", type=int, default=None)
    ap.add_argument("--chunks", type=int, default=None)
    ap.add_argument("--seed", type=int, default=0x5EED02)
    ap.add_argument("--k", type=int, default=REGEXP_K,
                    help="--workload regexp: the k of (a|b)*a(a|b){k} (the paper's regexp family)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-dfa", action="store_true")
    ap.add_argument("--no-counts", action="store_true", help="skip the host transition counters")
    ap.add_argument("--no-cpu-context", action="store_true",
                    help="skip the host recognition (serial table loop, chunks on all host threads)")
    ap.add_argument("--nfa", action="store_true",
                    help="also time the NFA variant of the classic algorithm (Sec. 2) on the same text "
                         "and count its transitions (Table 3's NFA columns)")
    ap.add_argument("--ablation", action="store_true",
                    help="also time the unminimised interface (every NFA state a slot)")
    ap.add_argument("--table-mode", type=int, default=0,
                    help="reach-kernel table layout (0 auto, 1 compact, 2 rep16, 3 rep32)")
    ap.add_argument("--piece-len", type=int, default=0,
                    help="intra-chunk speculation piece length (0 auto, 1 off, >= 64 bytes)")
    ap.add_argument("--probe", type=int, default=0,
                    help="bytes between convergence checks of the speculative runs (0 auto)")
    ap.add_argument("--text-path", type=int, default=0,
                    help="converged-phase text reads (0 auto, 1 global loads, 3 cooperative staging, 4 two chunks per lane, 5 set path)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist

    import paper_2412_14975_gb300 as lib
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(dev))

    name = args.workload
    stream = torch.cuda.current_stream()
    if name == "batch":
        run_batch(args, lib, torch, dev, stream, world, rank)
        if world > 1:
            dist.destroy_process_group()
        return
    if name == "served":
        run_served(args, lib, torch, dev, rank)
        if world > 1:
            dist.destroy_process_group()
        return
    desc, n_default, c_default = WORKLOADS[name]
    n_req = args.text_bytes or n_default
    c = args.chunks or c_default
    re_src = workload_re(name, args.k)
    prog = lib.ridfa_compile(re_src)
    info = prog.info
    d_text = make_text(name, n_req, args.seed + rank, dev)
    n = d_text.numel()
    c = min(c, n)
    stream = torch.cuda.current_stream()
    d_accept = torch.zeros(1, dtype=torch.uint8, device=dev)

    def step_dfa():
        lib.ridfa_recognize_dfa_async(prog, d_text, n, c, d_accept, stream=stream)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        if world > 1:
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
            dist.barrier()
        return ms

    # chunk-count autotuning (untimed): a few launch shapes matched to the resident lanes of the
    # GPU; the timed region below uses the winner
    autotune = None
    if args.chunks is None and n >= (1 << 24):
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        cands = sorted({c_default, 1 << 17, 1 << 18, sms * 1024, sms * 2048})
        autotune = {}
        for cc in cands:
            cc = min(cc, n)
            for _ in range(2):
                lib.ridfa_recognize_async(prog, d_text, n, cc, d_accept, stream=stream)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                lib.ridfa_recognize_async(prog, d_text, n, cc, d_accept, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            autotune[cc] = round(3 * n / (e0.elapsed_time(e1) / 1e3) / 1e9, 1)
        c = max(autotune, key=autotune.get)

    # correctness guard of the timed configuration (device result vs the synchronous API)
    acc = lib.ridfa_recognize(prog, d_text, n, c, stream=stream)

    tuning = {"table_mode": args.table_mode, "text_path": args.text_path, "piece_len": args.piece_len,
              "probe_interval": args.probe}

    def step_rid():
        lib.ridfa_recognize_async(prog, d_text, n, c, d_accept, tuning=tuning, stream=stream)

    with ClockSampler(local) as clk:      # sampling spans the warm-up and the timed steps
        ms = timed(step_rid, args.steps, args.warmup)
    clocks = clk.summary()
    value = world * n * args.steps / (ms / 1e3) / 1e9

    dfa_value = None
    if not args.no_dfa and info["n_dfa_states"] and info["n_dfa_states"] <= lib.RIDFA_MAX_SLOTS:
        dacc = lib.ridfa_recognize_dfa(prog, d_text, n, c, stream=stream)
        assert dacc == acc, "RID and all-states DFA disagree"
        dms = timed(step_dfa, args.steps, args.warmup)
        dfa_value = world * n * args.steps / (dms / 1e3) / 1e9

    # roofline of the dominant kernel (reach): events around its launch on the same stream
    reach = []
    joins = []
    for _ in range(5):
        lib.ridfa_recognize_async(prog, d_text, n, c, d_accept,
                                  tuning={"profile": 1, "table_mode": args.table_mode,
                                          "text_path": args.text_path, "piece_len": args.piece_len,
                                          "probe_interval": args.probe}, stream=stream)
        r, j = lib.ridfa_last_timings(prog)
        reach.append(r)
        joins.append(j)
    reach_ms = statistics.median(reach)
    join_ms = statistics.median(joins)
    alg_bytes = n + c * info["k"] * 2 + c * 4
    peaks, peak_kind = measured_peaks()
    achieved = alg_bytes / (reach_ms / 1e3) / 1e9
    # the second roof: the converged step's two lane-private shared-memory gathers per byte,
    # measured on this GPU by the library's microbenchmark
    lut_rate = lib.ridfa_bench_smem_gather(1 << 16) / 1e9
    text_rate = n / (reach_ms / 1e3) / 1e9
    traffic = None
    if name == REACH_TRAFFIC["workload"] and args.table_mode == 0 and args.text_path == 0 and c == 155648:
        traffic = int(REACH_TRAFFIC["dram_bytes_per_text_byte"] * n)
    roofline = {"bound": "hbm", "achieved": round(achieved, 2), "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": traffic,
                "kernel": "rid_reach_kernel", "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": alg_bytes, "kernel_ms": round(reach_ms, 4),
                "join_ms": round(join_ms, 4),
                "smem_gather": {"peak_text_GBps": round(lut_rate, 1), "achieved_text_GBps": round(text_rate, 1),
                                "frac": round(text_rate / lut_rate, 4),
                                "note": "ridfa_bench_smem_gather: 2 lane-private gathers per byte, all SMs"}}

    # the NFA variant (Sec. 2): every position-NFA state a start state, sets simulated per start
    nfa = None
    if args.nfa and info["n_nfa"] <= 128:
        assert lib.ridfa_recognize_nfa(prog, d_text, n, c, stream=stream) == acc, "RID and NFA variant disagree"
        k_nfa = 3
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k_nfa):
            lib.ridfa_recognize_nfa(prog, d_text, n, c, stream=stream)
        nfa = {"value": round(n * k_nfa / (time.perf_counter() - t0) / 1e9, 3), "unit": "GB/s",
               "note": "ridfa_recognize_nfa, synchronous calls (reach + composition join + accept read back)"}

    # the effect of interface minimisation (Sec. 3.4): the same text with I^B = every singleton
    ablation = None
    if args.ablation:
        pu = lib.ridfa_compile(re_src, minimize_interface=False, build_dfa=False)
        if pu.info["k"] <= lib.RIDFA_MAX_SLOTS:
            def step_unmin():
                lib.ridfa_recognize_async(pu, d_text, n, c, d_accept, stream=stream)
            assert lib.ridfa_recognize(pu, d_text, n, c, stream=stream) == acc
            ums = timed(step_unmin, max(3, args.steps // 2), args.warmup)
            ablation = {"unminimized_k": pu.info["k"], "minimized_k": info["k"],
                        "unminimized_GBps": round(world * n * max(3, args.steps // 2) / (ums / 1e3) / 1e9, 3)}

    e2e = None
    if not args.no_e2e:
        h_text = torch.empty(n, dtype=torch.uint8, pin_memory=True)
        h_text.copy_(d_text)
        d_in = torch.empty_like(d_text)
        for _ in range(2):
            assert lib.ridfa_recognize_host(prog, h_text, n, c, d_in, stream=stream) == acc
        k = max(3, min(args.steps, 10))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k):
            # one C-ABI call: host-to-device copy of the text, reach, join, accept byte back
            lib.ridfa_recognize_host(prog, h_text, n, c, d_in, stream=stream)
        dt = time.perf_counter() - t0
        e2e = {"value": round(n * k / dt / 1e9, 3), "unit": "GB/s", "h2d_bytes_per_step": n,
               "d2h_bytes_per_step": 1}
        del d_in

    # work of the timed configuration, counted on the host by the library's counter tool:
    # W_conv (lookups with merged runs, the kernel's algorithmic work) and the paper's W_paper,
    # for the RID and for the all-states DFA (the transition ratio of the paper's Table 3)
    work = None
    if rank == 0 and not args.no_counts:
        hx = h_text.numpy() if not args.no_e2e else d_text.cpu().numpy()
        t0 = time.perf_counter()
        rc = lib.ridfa_count_transitions(prog, hx, c)
        work = {"rid_w_conv_per_byte": round(rc["w_conv"] / n, 5),
                "rid_w_paper_per_byte": round(rc["w_paper"] / n, 5),
                "rid_runs": rc["runs"], "rid_dead_runs": rc["dead_runs"],
                "rid_converge_hist_log2": rc["converge_hist"]}
        if info["n_dfa_states"]:
            dc = lib.ridfa_count_transitions(prog, hx, c, dfa=True)
            work.update({"dfa_w_conv_per_byte": round(dc["w_conv"] / n, 5),
                         "dfa_w_paper_per_byte": round(dc["w_paper"] / n, 5),
                         "transition_ratio_dfa_over_rid": round(dc["w_paper"] / max(rc["w_paper"], 1), 4)})
        if args.nfa and info["n_nfa"] <= 128:
            nc = lib.ridfa_count_transitions(prog, hx, c, nfa=True)
            work.update({"nfa_w_paper_per_byte": round(nc["w_paper"] / n, 5),
                         "transition_ratio_nfa_over_rid": round(nc["w_paper"] / max(rc["w_paper"], 1), 4)})
        work["count_s"] = round(time.perf_counter() - t0, 2)
        lpb = 1 + rc["w_conv"] / n
        roofline["smem_gather"]["lookups_per_byte"] = round(lpb, 5)
        # the binding roof: the slower of the text at HBM bandwidth and the lookups at the
        # measured gather rate (the microbenchmark does 2 lookups per byte)
        lut_text_rate = lut_rate * 2.0 / lpb
        roofline["smem_gather"]["roof_text_GBps"] = round(lut_text_rate, 1)
        roofline["smem_gather"]["roof_frac"] = round(text_rate / lut_text_rate, 4)
        hbm_text_rate = peaks["hbm_gbs"] * n / alg_bytes
        roofline["binding"] = "smem_lookups" if lut_text_rate < hbm_text_rate else "hbm"
        roofline["binding_frac"] = round(text_rate / min(lut_text_rate, hbm_text_rate), 4)
    # the paper's own setting for context: the same recognition on the host's cores through the
    # library's host entry point (serial table loop; one chunk per hardware thread)
    cpu_context = None
    if rank == 0 and world == 1 and not args.no_cpu_context:
        hx = h_text.numpy() if not args.no_e2e else d_text.cpu().numpy()
        cpu_context = measure_cpu_context(lib, prog, hx, acc, info["n_dfa_states"] > 0)
    if not args.no_e2e:
        del h_text

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(name, re_src)

    # the other two numbers of the metric, on the same GPU in the same run (one GPU only: under
    # torchrun every rank measures its single-text replica alone)
    batched = served = None
    if name == "c3" and world == 1 and args.text_bytes is None:
        del d_text
        torch.cuda.empty_cache()
        if not args.no_batched:
            batched = measure_batch(args, lib, torch, dev, stream, world, rank,
                                    args.combined_batch_steps, args.warmup)
            torch.cuda.empty_cache()
        if not args.no_served:
            served = measure_served(args, lib, torch, dev, rank,
                                    [int(r) for r in args.combined_served_rates.split(",")],
                                    args.combined_served_seconds)

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
                "config": {"workload": f"{name}: {desc}", "text_bytes": n, "n_chunks": c,
                           "re": re_src, "nfa_states": info["n_nfa"], "ridfa_states": info["n_states"],
                           "k": info["k"], "classes": info["n_classes"],
                           "dfa_states": info["n_dfa_states"], "accept": bool(acc),
                           "l2": "inputs larger than L2 (text > 129 MB), no flush",
                           "chunk_autotune_GBps": autotune,
                           "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
                "dfa_value": round(dfa_value, 3) if dfa_value else None,
                "roofline": roofline, "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu,
                "cpu_context": cpu_context, "work": work,
                "interface_ablation": ablation, "nfa_variant": nfa,
                "batched": batched, "served": served,
                "gpu_launches": 2 * args.steps}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
