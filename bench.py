"""Benchmark of EP-HDC client-side encrypted inference on one GB300 per rank.

A step is one pass of the whole client path over one batch of synthetic queries:
HDC projection + quantisation, BFV batch encoding (slot packing, inverse NTT mod
t, lift, NTT per limb), plaintext x ciphertext multiply-accumulate against the
device-resident encrypted model, rotate-and-sum with key switching, and the
inverse NTT of the score ciphertexts.  The encrypted model and the rotation keys
are made once before timing (server side, not part of the client path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload face1024]
  python bench.py --impl reference ...   (the CPU oracle on the host cores)

Under torchrun every rank runs an independent replica (the path has no exchange
step), so the value is the queries of all ranks over the slowest rank's time.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "encrypted HDC queries/sec (D=10000, n=8192) and % HBM/INT8 roofline vs plain"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="face1024")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-perquery", action="store_true")
    ap.add_argument("--clientrt-table", action="store_true",
                    help="only print the client-runtime table at the paper's parameters")
    ap.add_argument("--no-sr", action="store_true",
                    help="skip the client-runtime comparison with the server-side variant")
    ap.add_argument("--cpu-budget-s", type=float, default=20.0)
    ap.add_argument("--serve-requests", type=int, default=20000)
    ap.add_argument("--streams", type=int, default=4,
                    help="streams (contexts) that consecutive batches alternate over")
    ap.add_argument("--mac-mode", type=int, default=-1,
                    help="force the multiply-accumulate schedule (profiling)")
    ap.add_argument("--hdc-mode", type=int, default=-1,
                    help="force the HDC projection kernel (library default otherwise)")
    ap.add_argument("--mac-tile", type=int, default=-1,
                    help="force the tiled multiply-accumulate with this tiling (profiling)")
    ap.add_argument("--pack", type=int, default=0,
                    help="consecutive batches packed into one step (one model stream); "
                         "0 = as many as fit in 16 query groups")
    ap.add_argument("--dim", type=int, default=0,
                    help="override the hypervector dimension D (profiling of smaller cases)")
    ap.add_argument("--batch", type=int, default=0,
                    help="override the workload's batch size (profiling of smaller cases)")
    ap.add_argument("--layout", type=int, default=-1,
                    help="storage layout of plaintexts and model (0 standard, 1 "
                         "coefficient-blocked); default 0")
    ap.add_argument("--chunk", type=int, default=0,
                    help="encode and accumulate this many plaintext indices of every group "
                         "at a time (0 = the whole pass at once)")
    ap.add_argument("--compact", action="store_true",
                    help="the compact model: c0 stored, c1 regenerated by the tiled MAC")
    ap.add_argument("--model-digits", type=int, default=-1,
                    help="1: the digit model (fp16 operand of the model's signed digits, read "
                         "by the digit-outer-product tensor-core MAC), 0: residues; default: "
                         "digits for dense65536, dense65536_r8 and clients64")
    ap.add_argument("--no-legs", action="store_true",
                    help="time only the headline workload (not clients64, serve, dense65536)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------------ CPU oracle leg
def oracle_units(w, B, units, seed):
    """Time the oracle's client path on `units` plaintext indices (D-chunks) of one
    batch of B queries, and separately its per-batch tail (rotate-and-sum).  Returns
    (seconds for the units, seconds for the tail, threads)."""
    import oracle as O
    from paper_2511_00737_gb300 import workload as WL
    Dsub = min(w.D, units * w.r)
    osub = O.Oracle(w.n, w.L, w.k, w.k_in, w.r, Dsub)
    X = WL.features(seed, B, w.F)
    Wt = WL.projection(seed, w.D, w.F)[:Dsub]
    cls = WL.classes(seed, w.k, w.D)[:, :Dsub]
    s, gk = osub.keygen(seed)
    model = osub.encrypt_model(seed, np.ascontiguousarray(cls), s)  # setup, not timed
    t0 = time.perf_counter()
    H = O.hdc_encode(X, np.ascontiguousarray(Wt), w.shift, w.bits)
    m = osub.encode_plain(H)
    acc = osub.ptct_mac(m, B, model)
    t1 = time.perf_counter()
    osub.rotate_sum(gk, acc)
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1, O.num_threads()


def cpu_baseline(w, B, budget_s, seed):
    import oracle as O
    P = -(-w.D // w.r)
    # calibrate on one unit, then size the sample to the budget
    t_one, t_tail, cores = oracle_units(w, B, 1, seed)
    units = int(max(1, min(P, budget_s / max(t_one, 1e-3))))
    t_units, t_tail, cores = oracle_units(w, B, units, seed)
    est = t_units * P / units + t_tail
    return {"value": B / est, "unit": "queries/s", "cores": cores, "kind": "oracle",
            "sample": "%d of %d plaintext indices of one %d-query batch (%.1f s) plus the "
                      "rotate-and-sum tail (%.2f s), scaled to the full batch" % (
                          units, P, B, t_units, t_tail)}


def run_reference(args, w, B):
    rank, _, world = dist_env()
    if rank != 0:
        return
    import oracle as O
    P = -(-w.D // w.r)
    budget = max(0.02, 150.0 / max(1, args.steps + args.warmup))
    t_one, t_tail, cores = oracle_units(w, B, 1, w.seed)
    units = int(max(1, min(P, budget / max(t_one, 1e-3))))
    for _ in range(args.warmup):
        oracle_units(w, B, units, w.seed)
    tot = 0.0
    for _ in range(args.steps):
        t, _, cores = oracle_units(w, B, units, w.seed)
        tot += t
    per_unit = tot / (args.steps * units)
    est = per_unit * P + t_tail
    value = B / est
    line = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": est * 1000.0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "impl": "reference",
            "config": config_of(w, B),
            "cpu_baseline": {"value": value, "unit": "queries/s", "cores": cores,
                             "kind": "oracle",
                             "sample": "%d of %d plaintext indices per step, %d steps, plus the "
                                       "rotate-and-sum tail" % (units, P, args.steps)},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(w, B, per_step=None):
    return {"workload": "%s: B=%d queries, F=%d, D=%d, %d-bit HVs, k=%d classes, BFV n=%d, "
                        "t=65537, L=%d x 30-bit primes, layout k_in=%d r=%d" % (
                            w.name, B, w.F, w.D, w.bits, w.k, w.n, w.L, w.k_in, w.r),
            "global_batch": per_step or B, "n": w.n, "L": w.L, "D": w.D, "F": w.F, "k": w.k,
            "hv_bits": w.bits, "k_in": w.k_in, "r": w.r,
            "l2": "inputs larger than L2: the encrypted model streamed every step is "
                  "larger than the 129 MB L2", "parallelism": "replicas"}


# ------------------------------------------------------------------ parity of the timed work
DIGESTS = {"face1024": "face1024x16", "clients64": "clients64", "dense65536": "dense65536"}
DIGIT_WORKLOADS = ("dense65536", "dense65536_r8", "clients64")


def digest_check(out, ctx, name):
    """Compares query groups of the score ciphertexts in `out` (coefficient domain,
    [G][k/k_in][2][L][n]) word for word with the SHA-256 digests of the oracle's
    ciphertexts stored in tests/golden/<name>_group_digests.txt (written by the
    committed script beside it, which runs only the oracle)."""
    import hashlib
    path = os.path.join(ROOT, "tests", "golden", name + "_group_digests.txt")
    words = out.cpu().numpy().view(np.uint32).reshape(-1, ctx.Kp, 2, ctx.L, ctx.n)
    groups, ok = [], True
    for line in open(path):
        if not line.strip() or line.startswith("#"):
            continue
        g, _, _, digest = line.split()
        got = np.ascontiguousarray(words[int(g)], dtype="<u4")
        ok = ok and hashlib.sha256(got.tobytes()).hexdigest() == digest
        groups.append(int(g))
    return {"checked": "score ciphertexts of groups %s vs oracle digests (%s)" % (
        groups, os.path.basename(path)), "match": bool(ok)}


# ------------------------------------------------------------------ our arm
def run_ours(args, w, B):
    import torch
    from paper_2511_00737_gb300 import ephdc as E
    from paper_2511_00737_gb300 import workload as WL

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    seed = w.seed + 7919 * rank
    multi = bool(w.clients)
    cap = 2 * ((w.n // (2 * w.r)) // w.k_in)
    # a step packs `pack` consecutive batches of the workload into one pass, so the
    # encrypted model is streamed once for all of their groups
    groups_per_batch = -(-B // cap)
    batch = B
    pack = 1 if multi else (args.pack if args.pack > 0 else max(1, 16 // groups_per_batch))
    B = batch * pack
    if multi:
        from paper_2511_00737_gb300 import autotune as AT
        from paper_2511_00737_gb300 import batching as BT
    # packed multi-client steps replay whole groups, so reserve full groups
    ctx = E.Context.for_workload(w, max_batch=(-(-B // cap) * cap) if multi else B)
    # storage layout of plaintexts and model (standard unless forced: at dense65536 the
    # blocked layout's faster tensor-core product is offset by the encoder's scattered
    # 16-byte stores)
    layout = max(0, args.layout)
    ctx.tune_set("layout", layout)
    # the compact model: only c0 stored, c1 regenerated by the multiply-accumulate
    model_seed = seed if args.compact else -1
    ctx.tune_set("model_seed", model_seed)
    # the digit model (the model's signed base-256 digits as the tensor-core operand):
    # by default where many groups share each model read and k/k_in fills the MMA rows
    # (dense65536: MAC 15.5 ms vs 30.4 ms; clients64: 3.4 ms vs 4.2 ms), residues for the
    # 4-output face1024 step
    mdig = args.model_digits if args.model_digits >= 0 else int(w.name in DIGIT_WORKLOADS)
    ctx.tune_set("model_digits", mdig)
    if args.mac_mode >= 0:
        ctx.tune_set("mac_mode", args.mac_mode)
    if args.hdc_mode >= 0:
        ctx.tune_set("hdc_mode", args.hdc_mode)
    sk, gk = ctx.keygen(seed)
    cls = torch.from_numpy(WL.classes(seed, w.k, w.D)).to(dev)
    model = ctx.encrypt_model(cls, sk, seed)
    Wt = torch.from_numpy(WL.projection(seed, w.D, w.F)).to(dev)
    R = 4
    if multi:
        # each step packs the 64 clients' batches; R rotating sets of features
        Xh = [[torch.from_numpy(WL.features(seed, b, w.F, batch=1000 * s + i)).pin_memory()
               for i, b in enumerate(w.clients)] for s in range(R)]
        Xd = [[x.to(dev) for x in xs] for xs in Xh]
        pipe = BT.GraphedPipeline(ctx, Wt, model, gk, max_groups=ctx.groups(B))
        hdc = {}
        if args.hdc_mode < 0:  # the HDC projection kernel, timed on this batch
            hdc, _, _ = AT.tune_hdc(ctx, torch.cat(Xd[0]), Wt, reps=3)
        pt0 = ctx.encode_plain(ctx.hdc_encode(torch.cat(Xd[0]), Wt))
        if args.mac_mode >= 0:
            tuned = {"mac_mode": args.mac_mode}
        else:
            tuned, tuned_ms, _ = AT.tune_similarity(ctx, pt0, B, model, gk, reps=3)
        del pt0
        out = pipe.out
        enc, _, _ = AT.tune_encode(ctx, ctx.hdc_encode(torch.cat(Xd[0]), Wt), reps=3)
        tuned = {**tuned, **enc, **hdc}
        # consecutive steps alternate over S pipelines (each its own context, graphs and
        # stream, sharing the model and keys), so one step's MAC and rotations overlap
        # the next step's encoding
        S = max(1, args.streams)
        ctxs = [ctx] + [E.Context.for_workload(w, max_batch=ctx.groups(B) * cap)
                        for _ in range(S - 1)]
        for cx in ctxs[1:]:
            cx.tune_set("layout", layout)
            cx.tune_set("model_seed", model_seed)
            cx.tune_set("model_digits", mdig)
            AT.apply(cx, tuned)
        pipes = [pipe] + [BT.GraphedPipeline(cx, Wt, model, gk, max_groups=ctx.groups(B))
                          for cx in ctxs[1:]]
        for p_ in pipes:
            p_.graph(ctx.groups(B))   # captured before timing
        streams = [torch.cuda.Stream(device=dev) for _ in range(S)]
        outs = [p_.out for p_ in pipes]

        def step(i):
            pipes[i % S].launch(Xd[i % R], streams[i % S])
    else:
        Xh = [torch.from_numpy(WL.features(seed, B, w.F, batch=b)).pin_memory() for b in range(R)]
        Xd = [x.to(dev) for x in Xh]
        out = ctx.out_ct(B)
        from paper_2511_00737_gb300 import autotune as AT
        hdc = {}
        if args.hdc_mode < 0:  # the HDC projection kernel, timed on this batch
            hdc, _, _ = AT.tune_hdc(ctx, Xd[0], Wt, reps=5)
        H0 = ctx.hdc_encode(Xd[0], Wt)
        tuned, _, _ = AT.tune_encode(ctx, H0, reps=5)  # pass schedule of the transforms
        tuned = {**tuned, **hdc}
        if args.mac_tile >= 0:
            tuned = {**tuned, "mac_mode": 2, "mac_tile": args.mac_tile}
            AT.apply(ctx, tuned)
        elif ctx.groups(B) >= 2 and args.mac_mode < 0:
            # several groups share each model read: let the autotuner pick the schedule
            pt0 = ctx.encode_plain(H0)
            mac, _, _ = AT.tune_similarity(ctx, pt0, B, model, gk, reps=2)
            tuned = {**tuned, **mac}
            del pt0
        del H0
        # consecutive batches alternate over S streams, each with its own context
        # (scratch) and output, sharing the resident model and keys, so one batch's
        # latency-bound rotations overlap the next batch's encoding and MAC
        S = max(1, args.streams)
        ctxs = [ctx] + [E.Context.for_workload(w, max_batch=B) for _ in range(S - 1)]
        for cx in ctxs[1:]:
            cx.tune_set("layout", layout)  # the shared model's layout and form
            cx.tune_set("model_seed", model_seed)
            cx.tune_set("model_digits", mdig)
            if tuned:
                AT.apply(cx, tuned)
        for cx in ctxs:
            cx.tune_set("chunk", args.chunk)
            if args.hdc_mode >= 0:
                cx.tune_set("hdc_mode", args.hdc_mode)
        outs = [out] + [cx.out_ct(B) for cx in ctxs[1:]]
        streams = [torch.cuda.Stream(device=dev) for _ in range(S)]

        def step(i):
            j = i % S
            with torch.cuda.stream(streams[j]):
                ctxs[j].infer(Xd[i % R], Wt, model, gk, out=outs[j])
    out_h = torch.empty(out.shape, dtype=out.dtype).pin_memory()
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_2511_00737_gb300 import replicas as RP

    def maxall(v):
        return RP.max_over_ranks(v, device=dev)

    st = torch.cuda.current_stream()
    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    ctx.profile(True)
    ctx.profile_read()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    all_ctx = ctxs
    side = streams
    for cx in all_ctx:
        cx.profile(True)
        cx.profile_read()
    e0.record(st)
    for s_ in side:
        s_.wait_stream(st)
    for i in range(args.steps):
        step(i)
    for s_ in side:
        st.wait_stream(s_)
    e1.record(st)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    def read_stages():
        sm_, sc_, ln_ = {}, {}, 0
        for cx in all_ctx:
            a, b_, c_ = cx.profile_read()
            for k in a:
                sm_[k] = sm_.get(k, 0.0) + a[k]
                sc_[k] = sc_.get(k, 0) + b_[k]
            ln_ += c_
        return sm_, sc_, ln_

    stage_ms, stage_calls, launches = read_stages()
    # the timed work's own output: the last timed step on stream 0 used feature set
    # last % R; with the digests' inputs (set 0 of the rank-0 seed) check it
    parity = None
    can_check = (rank == 0 and not args.dim and not args.batch and w.name in DIGESTS and
                 not args.compact and
                 (multi or (w.name != "face1024" or (batch == 1024 and pack == 16))))
    if can_check and not multi:
        last = max(i for i in range(args.steps) if i % S == 0)
        if last % R == 0:
            parity = digest_check(outs[0], ctx, DIGESTS[w.name])
            parity["step"] = "timed step %d (stream 0)" % last
    roof_pass = "the timed region"
    if not multi and S > 1:
        # overlapping batches stretch each kernel's event time: take the per-stage
        # breakdown and the roofline from a single-stream pass of the same steps
        k1 = min(args.steps, 200)
        for i in range(k1):
            ctx.infer(Xd[i % R], Wt, model, gk, out=out)
        torch.cuda.synchronize()
        one_ms, one_calls, _ = read_stages()
        stage_ms = {k: v * args.steps / k1 for k, v in one_ms.items()}
        stage_calls = {k: v * args.steps // k1 for k, v in one_calls.items()}
        roof_pass = "a single-stream pass of %d steps after the timed region" % k1
    if multi:
        # graph replays record no stage events: take the stage breakdown and the
        # launches per step from a few eager steps of the same packed work on one stream
        read_stages()
        ksteps_eager = 5
        pipe.use_graphs = False
        for i in range(ksteps_eager):
            pipe.launch(Xd[i % R], streams[0])
        torch.cuda.synchronize()
        stage_ms, stage_calls, launches = read_stages()
        stage_ms = {k: v * args.steps / ksteps_eager for k, v in stage_ms.items()}
        stage_calls = {k: v * args.steps // ksteps_eager for k, v in stage_calls.items()}
        launches = launches * args.steps // ksteps_eager
        pipe.use_graphs = True
        roof_pass = "%d eager single-stream steps after the timed region" % ksteps_eager
        if can_check:
            res, _ = pipe.run(Xd[0])   # the timed step's graph on feature set 0
            torch.cuda.synchronize()
            parity = digest_check(res, ctx, DIGESTS[w.name])
            parity["step"] = "one graph-replayed step on feature set 0 after the timed region"
    for cx in all_ctx:
        cx.profile(False)
    value, ms_total = RP.job_throughput(B * args.steps, e0.elapsed_time(e1), world, device=dev)
    ms = ms_total / args.steps

    # end to end: pinned host inputs in, score ciphertexts back to pinned host
    ksteps = max(1, min(args.steps, 300))
    out_hs = [out_h] + [torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in outs[1:]]
    barrier()
    torch.cuda.synchronize()
    e0.record(st)
    for s_ in side:
        s_.wait_stream(st)
    for i in range(ksteps):
        if multi:
            j = i % S
            with torch.cuda.stream(streams[j]):
                for xd, xh in zip(Xd[i % R], Xh[i % R]):
                    xd.copy_(xh, non_blocking=True)
                res, _ = pipes[j].launch(Xd[i % R], streams[j])
                out_hs[j][:res.numel()].copy_(res, non_blocking=True)
        else:
            j = i % S
            with torch.cuda.stream(streams[j]):
                Xd[i % R].copy_(Xh[i % R], non_blocking=True)
                ctxs[j].infer(Xd[i % R], Wt, model, gk, out=outs[j])
                out_hs[j].copy_(outs[j], non_blocking=True)
    for s_ in side:
        st.wait_stream(s_)
    e1.record(st)
    torch.cuda.synchronize()
    barrier()
    ms_e2e = maxall(e0.elapsed_time(e1)) / ksteps
    e2e = {"value": world * B / (ms_e2e / 1000.0), "unit": "queries/s",
           "h2d_bytes_per_step": int(B * w.F), "d2h_bytes_per_step": int(out.numel() * 4),
           "ms_per_step": ms_e2e}

    # the per-query GPU form: one query per call, packed so that log2(n/(2 k_in))
    # rotations fold the whole hypervector (the dense shape of HE-HDC)
    perq = None
    if not args.no_perquery and rank == 0 and not multi:
        perq = per_query_form(w, dev)

    # client runtime against the server-side variant, on one batch of at most 4 groups
    clrt = None
    if not args.no_sr and rank == 0 and not multi:
        clrt = client_runtime(w, dev, min(batch, 4 * cap))

    # roofline of the dominant stage
    pk, src = peaks()
    # integer-pipe peaks of this device, measured by register-only kernels
    bfly_s, mac_s = E.ephdc_measure_int_peaks()
    pk = dict(pk, bfly_tps=bfly_s / 1e12, mac_tps=mac_s / 1e12)
    int_peaks = {"butterflies_T_per_s": bfly_s / 1e12, "mac64_T_per_s": mac_s / 1e12,
                 "source": "ephdc_measure_int_peaks, register-only kernels on this GPU"}
    dom = max(stage_ms, key=lambda s: stage_ms[s])
    roof = roofline(ctx, w, B, dom, stage_ms, stage_calls, pk, src)
    roof["measured_in"] = roof_pass
    roof["int_peaks"] = int_peaks

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, batch, args.cpu_budget_s, seed)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "u32", "data": "synthetic", "config": config_of(w, batch, B),
                "clocks": clk, "e2e": e2e, "gpu_launches": int(launches),
                "roofline": roof, "cpu_baseline": cpu,
                "stages_ms_per_step": {k: v / max(1, args.steps) for k, v in stage_ms.items()},
                "per_query_form": perq, "client_runtime_vs_server_side": clrt,
                "parity": parity}
        if not multi:
            line["config"]["streams"] = S
            if args.chunk:
                line["config"]["chunk_plaintexts"] = args.chunk
            line["config"]["batches_per_step"] = pack
            line["config"]["batch"] = batch
        line["config"]["storage_layout"] = "coefficient-blocked" if layout else "standard"
        if args.compact:
            line["config"]["model"] = ("compact: c0 stored, c1 regenerated from the seed by "
                                       "the multiply-accumulate")
        if mdig:
            line["config"]["model"] = ("digit model: fp16 tensor-core operand of the signed "
                                       "base-256 digits")
        if not multi and tuned:
            line["config"]["mac_schedule"] = tuned
        if multi:
            line["config"]["streams"] = S
            line["config"]["clients"] = len(w.clients)
            line["config"]["mac_schedule"] = tuned
            line["config"]["cuda_graph"] = True
    for cx in ctxs:
        cx.close()
    if dist is not None:
        dist.destroy_process_group()
    return line if rank == 0 else None


def client_runtime(w, dev, B, reps=5):
    """Client cost of the client-side path vs the server-side variant (HE-HDC-SR) on
    one batch of the workload (Sec. 6, Table t:clientrt): EP-HDC's client encodes
    plaintexts and runs the HE compute; the HE-HDC-SR client encrypts its query
    plaintexts and decrypts the returned scores.  HDC encoding, common to both, is
    left out as in the paper's table.  Device milliseconds per batch, CUDA events on
    one stream, after a warm-up; each side's transforms at their fastest pass
    schedule."""
    import torch
    from paper_2511_00737_gb300 import ephdc as E
    from paper_2511_00737_gb300 import workload as WL
    ctx = E.Context.for_workload(w, max_batch=B)
    sk, gk = ctx.keygen(w.seed)
    cls = torch.from_numpy(WL.classes(w.seed, w.k, w.D)).to(dev)
    model = ctx.encrypt_model(cls, sk, w.seed)
    mm = ctx.encode_model_plain(cls)
    Wt = torch.from_numpy(WL.projection(w.seed, w.D, w.F)).to(dev)
    H = ctx.hdc_encode(torch.from_numpy(WL.features(w.seed, B, w.F)).to(dev), Wt)
    pt = ctx.encode_plain(H)
    ctq = ctx.encrypt_queries(H, sk, w.seed)
    out = ctx.out_ct(B)
    out_sr = ctx.out_ct(B)
    scores = torch.empty((B, w.k), dtype=torch.int32, device=dev)

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    # each side's transforms at its fastest pass schedule
    encpt, enc = float("inf"), float("inf")
    for plan in (0, 1, 2):
        ctx.tune_set("ntt_plan", plan)
        encpt = min(encpt, timed(lambda: E.bfv_encode_plain(ctx.ctx, H, B, pt)))
        enc = min(enc, timed(lambda: E.bfv_encrypt_queries(ctx.ctx, H, B, sk, w.seed, ctq)))
    he = timed(lambda: E.bfv_ptct_similarity(ctx.ctx, pt, B, model, gk, out))
    srv = timed(lambda: E.bfv_ctpt_similarity(ctx.ctx, ctq, B, mm, gk, out_sr))
    dec = timed(lambda: E.bfv_decrypt_scores(ctx.ctx, sk, out_sr, B, scores))
    same = bool(torch.equal(ctx.decrypt_scores(sk, out, B), ctx.decrypt_scores(sk, out_sr, B)))
    ctx.device_status()
    up = int(E.lib().ephdc_query_ct_bytes(ctx.ctx, B))
    down = int(E.lib().ephdc_out_ct_bytes(ctx.ctx, B))
    ctx.close()
    ep_ms, sr_ms = encpt + he, enc + dec
    return {"batch": B, "unit": "ms per batch",
            "client_side": {"client_ms": ep_ms, "encpt_ms": encpt, "he_compute_ms": he,
                            "message_bytes": down},
            "server_side": {"client_ms": sr_ms, "encrypt_ms": enc, "decrypt_ms": dec,
                            "server_ms": srv, "upload_bytes": up, "download_bytes": down},
            "client_speedup": sr_ms / ep_ms, "message_ratio": up / down,
            "same_scores": same}


def clientrt_table(dev, reps=10):
    """Table t:clientrt's four points at the paper's own parameters (Face: k = 2, the
    SIMD layout k_in = k, r = 1, one batch of N/2 queries; q at the 128-bit bound
    with 27-bit primes: 2 at N = 2048, 4 at N = 4096): client runtime of the
    client-side path (EncPt + HE compute) and of the server-side variant
    (encryption + decryption) on this GPU, and both message sizes."""
    import torch
    from paper_2511_00737_gb300 import ephdc as E
    from paper_2511_00737_gb300 import workload as WL
    rows = []
    for N, D in [(2048, 1024), (2048, 2048), (4096, 1024), (4096, 2048)]:
        L, F, seed = (2 if N == 2048 else 4), 608, 2511
        cap = N // 2
        ctx = E.Context(N, L, 2, 2, 1, D, F, 8, WL.default_shift(F, 8), cap, prime_bits=27)
        sk, gk = ctx.keygen(seed)
        cls = torch.from_numpy(WL.classes(seed, 2, D)).to(dev)
        model = ctx.encrypt_model(cls, sk, seed)
        Wt = torch.from_numpy(WL.projection(seed, D, F)).to(dev)
        H = ctx.hdc_encode(torch.from_numpy(WL.features(seed, cap, F)).to(dev), Wt)
        pt = ctx.encode_plain(H)
        ctq = ctx.encrypt_queries(H, sk, seed)
        mm = ctx.encode_model_plain(cls)
        out, out_sr = ctx.out_ct(cap), ctx.out_ct(cap)
        scores = torch.empty((cap, 2), dtype=torch.int32, device=dev)

        def timed(fn):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                fn()
            b.record()
            torch.cuda.synchronize()
            return a.elapsed_time(b) / reps

        encpt = timed(lambda: E.bfv_encode_plain(ctx.ctx, H, cap, pt))
        he = timed(lambda: E.bfv_ptct_similarity(ctx.ctx, pt, cap, model, gk, out))
        enc = timed(lambda: E.bfv_encrypt_queries(ctx.ctx, H, cap, sk, seed, ctq))
        E.bfv_ctpt_similarity(ctx.ctx, ctq, cap, mm, gk, out_sr)
        dec = timed(lambda: E.bfv_decrypt_scores(ctx.ctx, sk, out_sr, cap, scores))
        same = bool(torch.equal(ctx.decrypt_scores(sk, out, cap), ctx.decrypt_scores(sk, out_sr, cap)))
        rows.append({"N": N, "D": D, "L": L, "log2_q": round(sum(math.log2(q) for q in ctx.q), 1),
                     "batch": cap,
                     "client_side_ms": encpt + he, "encpt_ms": encpt, "he_compute_ms": he,
                     "client_side_message_bytes": int(E.lib().ephdc_out_ct_bytes(ctx.ctx, cap)),
                     "server_side_ms": enc + dec, "encrypt_ms": enc, "decrypt_ms": dec,
                     "server_side_message_bytes": int(E.lib().ephdc_query_ct_bytes(ctx.ctx, cap)),
                     "client_speedup": (enc + dec) / (encpt + he), "same_scores": same})
        ctx.device_status()
        ctx.close()
    return rows


def per_query_form(w, dev, queries=32):
    import torch
    from paper_2511_00737_gb300 import ephdc as E
    from paper_2511_00737_gb300 import workload as WL
    kin = w.k
    r = w.n // (2 * kin)
    r = 1 << int(math.log2(r))
    ctx = E.Context(w.n, w.L, w.k, kin, r, w.D, w.F, w.bits, w.shift, 1)
    sk, gk = ctx.keygen(w.seed)
    model = ctx.encrypt_model(torch.from_numpy(WL.classes(w.seed, w.k, w.D)).to(dev), sk, w.seed)
    Wt = torch.from_numpy(WL.projection(w.seed, w.D, w.F)).to(dev)
    X = torch.from_numpy(WL.features(w.seed, queries, w.F)).to(dev)
    out = ctx.out_ct(1)
    for i in range(3):
        ctx.infer(X[i:i + 1], Wt, model, gk, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(queries):
        ctx.infer(X[i:i + 1].contiguous(), Wt, model, gk, out=out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / queries
    ctx.close()
    return {"value": 1000.0 / ms, "unit": "queries/s", "ms_per_query": ms,
            "layout": "k_in=%d r=%d (%d rotations per query)" % (kin, r, int(math.log2(r)))}


# DRAM bytes (read + write) per launch of the dominant kernel from one ncu capture of
# the same kernel and launch shape (dram__bytes_read.sum + dram__bytes_write.sum):
# (workload, groups per launch, stage) -> bytes
NCU_TRAFFIC = {("face1024", 16, "encode_plain"): 2727000320}


def roofline(ctx, w, B, dom, stage_ms, stage_calls, pk, src):
    G = ctx.groups(B)
    P, Kp, L, n = ctx.P, ctx.Kp, ctx.L, ctx.n
    calls = max(1, stage_calls[dom])
    t = stage_ms[dom] / calls / 1000.0
    if dom == "mac" and G >= 2:
        # several groups per model read: a compute-bound multi-group contraction
        macs = G * P * 2 * Kp * L * n
        ach = macs / t / 1e12
        peak = alu_peak_tmac(pk)
        return {"kernel": "ptct_mac (multi-group, %d groups)" % G, "bound": "alu",
                "achieved": ach, "peak": peak, "unit": "Tmodmac/s", "frac": ach / peak,
                "traffic": None,
                "peak_source": "derived: 152 SMs x 64 32-bit integer multiply-adds per clock x "
                               "%.0f MHz / 2 multiply-adds per 64-bit carry-chain step" %
                               pk.get("sm_max_mhz", 2070.0),
                "measured_peak": pk["mac_tps"], "frac_of_measured": ach / pk["mac_tps"],
                "measured_peak_source": "register-only 64-bit carry-chain multiply-accumulates "
                                        "(ephdc_measure_int_peaks)",
                "ms_per_launch": t * 1000.0}
    if dom == "mac":
        model = P * Kp * 2 * L * n * 4
        pt = G * P * L * n * 4
        acc = G * Kp * 2 * L * n * 4
        byts = model + pt + acc
        ach = byts / t / 1e9
        return {"kernel": "ptct_mac (+split reduce)", "bound": "hbm", "achieved": ach,
                "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": ach / pk["hbm_gbs"],
                "traffic": None, "algorithmic_bytes": byts, "peak_source": src,
                "ms_per_launch": t * 1000.0}
    if dom == "encode_plain":
        # integer-pipe bound: butterflies per second against the issue limit
        bfly = G * P * (L + 1) * (n // 2) * int(math.log2(n))
        ach = bfly / t / 1e12
        peak = alu_peak_tbfly(pk)
        return {"kernel": "encode_plain", "bound": "alu", "achieved": ach,
                "peak": peak, "unit": "Tbutterfly/s", "frac": ach / peak,
                "traffic": NCU_TRAFFIC.get((w.name, G, "encode_plain")),
                "algorithmic_bytes": B * w.D + G * P * L * n * 4,
                "peak_source": "pipe model: the lazy Shoup butterfly is bound by the FMA-heavy "
                               "pipe (its multiplies); %.2f butterflies per SM cycle with that "
                               "pipe busy every cycle (ncu on the register-only butterfly loop: "
                               "95.4%% FMA-heavy active, 51.3%% ALU) x 152 SMs x %.0f MHz" % (
                                   BFLY_PER_SM_CYCLE, pk.get("sm_max_mhz", 2070.0)),
                "peak_old_derivation": 152 * 4 * 32 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 8 / 1e12,
                "measured_peak": pk["bfly_tps"], "frac_of_measured": ach / pk["bfly_tps"],
                "measured_peak_source": "register-only lazy Shoup butterflies "
                                        "(ephdc_measure_int_peaks)",
                "ms_per_launch": t * 1000.0}
    if dom == "hdc_encode":
        ops = 2.0 * B * w.F * w.D
        ach = ops / t / 1e12
        # exact fp16 x fp16 -> fp32 on the tensor cores: the fp16 dense rate equals bf16's
        return {"kernel": "hdc_encode", "bound": "tensor", "achieved": ach,
                "peak": pk["bf16_tflops"], "unit": "TFLOP/s", "frac": ach / pk["bf16_tflops"],
                "traffic": None, "peak_source": src + " (bf16 burst; fp16 has the same rate)",
                "ms_per_launch": t * 1000.0}
    return {"kernel": dom, "bound": "alu", "achieved": None, "peak": None, "unit": None,
            "frac": None, "traffic": None, "ms_per_launch": t * 1000.0}


# Butterflies per SM cycle of a lazy Shoup butterfly with the FMA-heavy pipe (which runs
# its integer multiplies) busy every cycle.  From one ncu capture of the register-only
# butterfly loop (k_bfly_peak, 4.08e10 butterflies, 2.59e7 SM cycles): that pipe 95.44%
# active at 3.254 T butterflies/s, i.e. 4.08e10 / (0.9544 x 2.59e7 x 152) per SM cycle.
# The ALU pipe was 51.3% active, so the FMA-heavy pipe binds.
BFLY_PER_SM_CYCLE = 4.0803e10 / (0.9544 * 25898462.62 * 152)


def alu_peak_tbfly(pk):
    mhz = pk.get("sm_max_mhz", 2070.0)
    return 152 * mhz * 1e6 * BFLY_PER_SM_CYCLE / 1e12


def alu_peak_tmac(pk):
    # 152 SMs x 64 32-bit integer multiply-adds per clock (half the 128 lanes); one
    # 64-bit carry-chain multiply-accumulate is 2 of them (mad.lo.cc, madc.hi)
    mhz = pk.get("sm_max_mhz", 2070.0)
    return 152 * 64 * mhz * 1e6 / 2 / 1e12


def run_serve(args, w):
    """Serving loop: Poisson arrivals (2000 requests/s), lognormal batch sizes (median
    32, max 8192), continuous batching over two pipeline slots of up to 8 groups."""
    import torch
    from paper_2511_00737_gb300 import ephdc as E
    from paper_2511_00737_gb300 import serving as SV
    from paper_2511_00737_gb300 import workload as WL

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    seed = w.seed + 7919 * rank
    keyctx = E.Context.for_workload(w, max_batch=1024)
    sk, gk = keyctx.keygen(seed)
    model = keyctx.encrypt_model(torch.from_numpy(WL.classes(seed, w.k, w.D)).to(dev), sk, seed)
    Wt = torch.from_numpy(WL.projection(seed, w.D, w.F)).to(dev)
    t, sizes = WL.arrivals(seed, args.serve_requests, rate_per_s=2000.0, median=32,
                           max_batch=8192)
    pool_rows = 65536
    pool = torch.from_numpy(WL.features(seed, pool_rows, w.F)).to(dev)
    offs = np.random.default_rng(seed).integers(0, pool_rows - 8192, len(sizes))
    make_X = lambda rid: pool[offs[rid]:offs[rid] + int(sizes[rid])]
    results = {}
    clk = None
    for name, scale in (("poisson_2000_rps", 1.0), ("all_at_once", 0.0)):
        srv = SV.Server(w, Wt, model, gk, slots=2, max_groups=8)
        srv.warm()
        clocks = ClockSampler(local)
        clocks.start()
        wall = srv.run(t, make_X, time_scale=scale)
        c = clocks.stop()
        clk = clk or c
        results[name] = srv.report(wall)
        for s_ in srv.slots:
            s_.ctx.close()
        del srv
        torch.cuda.synchronize()
    live = results["poisson_2000_rps"]
    offered = float(np.sum(sizes)) / float(t[-1])
    if rank == 0:
        line = {"metric": METRIC, "value": live["queries_per_s"], "unit": "queries/s",
                "n_gpus": world, "steps": live["steps"], "warmup": 0,
                "ms_per_step": 1e3 * live["wall_s"] / max(1, live["steps"]),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "u32", "data": "synthetic", "clocks": clk,
                "config": {"workload": "serve: %d requests, Poisson 2000 req/s, lognormal "
                                       "batch (median 32, max 8192), F=%d, D=%d, k=%d, n=%d, "
                                       "L=%d, layout k_in=%d r=%d; 2 slots x 8 groups" % (
                                           len(sizes), w.F, w.D, w.k, w.n, w.L, w.k_in, w.r),
                           "offered_queries_per_s": offered},
                "serving": results}
    keyctx.close()
    return line if rank == 0 else None


def main():
    args = parse()
    from paper_2511_00737_gb300 import workload as WL
    w = WL.config(args.workload)
    if args.batch:
        w.B = args.batch
        w.clients = []
    if args.dim:
        w.D = args.dim
    B = w.B
    if args.clientrt_table:
        import torch
        rows = clientrt_table(torch.device("cuda"))
        print(json.dumps({"table": "client runtime, client-side vs server-side HE (Table "
                                   "t:clientrt shape), device ms per batch", "rows": rows}),
              flush=True)
        return
    if args.impl == "reference":
        run_reference(args, w, B if B else 1024)
        return
    if args.workload == "serve" and not args.batch:
        line = run_serve(args, w)
    else:
        line = run_ours(args, w, B)
    _, _, world = dist_env()
    if (line is not None and args.workload == "face1024" and not args.batch and not args.dim
            and world == 1 and not args.no_legs):
        line["legs"] = run_legs(args)
    if line is not None:
        print(json.dumps(line), flush=True)


# the other workloads of the metric's parameters (D = 10000, n = 8192) and the dense
# one, each timed on its own after the headline (1 GPU only), with fewer steps
LEG_KEYS = ("value", "unit", "steps", "warmup", "ms_per_step", "config", "clocks", "e2e",
            "gpu_launches", "roofline", "stages_ms_per_step", "parity", "serving")


def run_legs(args):
    import copy
    import torch
    from paper_2511_00737_gb300 import workload as WL
    out = {}
    # (leg, workload, steps, plaintext chunk): the last leg times the headline step as a
    # chunked pass (96 plaintext indices of every group encoded and accumulated at a
    # time), the measured answer to whether keeping each chunk's plaintexts in L2 pays
    legs = (("clients64", "clients64", 50, 0), ("serve", "serve", 0, 0),
            ("dense65536", "dense65536", 5, 0), ("face1024_chunked96", "face1024", 100, 96),
            ("face1024_compact_model", "face1024", 100, -1))
    for name, wname, steps, chunk in legs:
        a = copy.copy(args)
        a.workload = wname
        a.steps = max(1, min(args.steps, steps))
        a.warmup = 3
        a.no_cpu_baseline = a.no_perquery = a.no_sr = True
        a.pack, a.mac_mode, a.mac_tile, a.hdc_mode = 0, -1, -1, -1
        a.chunk = max(0, chunk)
        a.compact = chunk < 0   # the compact-model leg
        w = WL.config(wname)
        t0 = time.perf_counter()
        try:
            line = run_serve(a, w) if wname == "serve" else run_ours(a, w, w.B)
        except Exception as ex:  # a failed leg is reported; the headline line still prints
            import traceback
            traceback.print_exc(file=sys.stderr)
            out[name] = {"error": "%s: %s" % (type(ex).__name__, str(ex)[:300]),
                         "wall_s": time.perf_counter() - t0}
            continue
        rec = {k: line[k] for k in LEG_KEYS if k in line}
        rec["wall_s"] = time.perf_counter() - t0
        if name == "serve":
            rec["steps"] = line["steps"]
        out[name] = rec
        torch.cuda.empty_cache()
    return out


if __name__ == "__main__":
    main()
