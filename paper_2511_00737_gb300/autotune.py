"""Autotuner of the multiply-accumulate schedule.

For one context and group count G it times every candidate schedule of
bfv_ptct_similarity on the device with CUDA events (the result never changes,
only the speed), applies the fastest and remembers it in a JSON cache keyed by
GPU, ring degree, limbs, layout and G.  Candidates: the streaming kernel split
over plaintext ranges (several split caps), and the tiled multi-group kernel with
2 or 4 groups and 4, 7 or 8 outputs per warp, 8 to 64 groups per CTA and 4 to 15
plaintexts per staged chunk, and the exact signed-digit product on the tensor cores
(the only candidate when the context stores plaintexts and model coefficient-blocked).
It also picks the encoder's pass schedule (tune_encode) and the HDC projection kernel
(tune_hdc) by timing each.
A context with the digit model has one product, the digit outer product on the tensor
cores; its candidates are the cluster sizes that share each model block.
"""
import json
import os

import torch

CACHE = os.environ.get("EPHDC_TUNE_CACHE",
                       os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tuning.json"))


def _key(ctx, G):
    name = torch.cuda.get_device_name(ctx.device).replace(" ", "_")
    return "%s|n%d|L%d|k%d|kin%d|r%d|G%d|lay%d|cm%d|md%d" % (
        name, ctx.n, ctx.L, ctx.k, ctx.k_in, ctx.r, G, ctx.tune_get("layout"),
        int(ctx.tune_get("model_seed") >= 0), ctx.tune_get("model_digits"))


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(d):
    tmp = CACHE + ".tmp.%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def candidates(ctx, G):
    O = 2 * ctx.Kp
    if ctx.tune_get("layout") == 1:
        return [{"mac_mode": 3}]   # the blocked layout is read by the tensor cores only
    if ctx.tune_get("model_digits") == 1:   # read by the digit outer product only
        blocks = -(-G // 16)
        return [{"mac_mode": 4, "mac_cluster": c} for c in (1, 2, 4) if c == 1 or c < 2 * blocks]
    compact = ctx.tune_get("model_seed") >= 0  # regenerated by the tiled kernel only
    if compact and G < 2:
        return [{"mac_mode": 2}]
    out = [] if compact else [{"mac_mode": 1, "mac_splits": s} for s in (0, 8, 16, 32)]
    if G >= 2 and O <= 32 and not compact:
        out.append({"mac_mode": 3})
    if G >= 2:
        for gt in (2, 4):
            for ot in (4, 7, 8):
                wo = -(-O // ot)
                for gc in (8, 16, 32, 64):
                    if gc % gt or (gc // gt) * wo > 16 or gc > 2 * G + gt:
                        continue
                    for ic in (4, 8, 15):
                        if 2 * ic * (gc + O) * 128 > 227 * 1024:
                            continue
                        out.append({"mac_mode": 2,
                                    "mac_tile": gt * 1000000 + ot * 10000 + gc * 100 + ic})
    return out


def apply(ctx, knobs):
    for k, v in knobs.items():
        ctx.tune_set(k, v)


def _time(fn, reps):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_similarity(ctx, pt, B, model, gk, reps=5, use_cache=True, max_candidates=None):
    """Pick the fastest MAC schedule for this batch size; returns (knobs, ms, table)."""
    G = ctx.groups(B)
    key = _key(ctx, G)
    cache = _load() if use_cache else {}
    if use_cache and key in cache:
        apply(ctx, cache[key]["knobs"])
        return cache[key]["knobs"], cache[key]["ms"], []
    out = ctx.out_ct(B)
    table = []
    cands = candidates(ctx, G)
    if max_candidates:
        cands = cands[:max_candidates]
    from .ephdc import EphdcError
    for knobs in cands:
        base = {"mac_mode": 0, "mac_splits": 0}
        try:
            apply(ctx, {**base, **knobs})
            ms = _time(lambda: ctx.ptct_similarity_into(pt, B, model, gk, out), reps)
        except EphdcError:
            # a schedule this device refuses to launch (a cluster it cannot place, a
            # tile over its shared memory) is skipped; the others are still timed
            continue
        table.append((ms, knobs))
    if not table:
        raise RuntimeError("no multiply-accumulate schedule could be launched")
    table.sort(key=lambda x: x[0])
    best_ms, best = table[0]
    apply(ctx, {"mac_mode": 0, "mac_splits": 0, **best})
    if use_cache:
        cache = _load()
        cache[key] = {"knobs": best, "ms": best_ms}
        _save(cache)
    return best, best_ms, table


def tune_encode(ctx, H, reps=5, use_cache=True):
    """Pick the fastest pass schedule of the encoding transforms for this batch."""
    B = H.shape[0]
    key = _key(ctx, ctx.groups(B)) + "|encode"
    cache = _load() if use_cache else {}
    if use_cache and key in cache:
        apply(ctx, cache[key]["knobs"])
        return cache[key]["knobs"], cache[key]["ms"], []
    table = []
    for v in (0, 1, 2):
        ctx.tune_set("ntt_plan", v)
        ms = _time(lambda: ctx.encode_plain(H), reps)
        table.append((ms, {"ntt_plan": v}))
    table.sort(key=lambda x: x[0])
    best_ms, best = table[0]
    apply(ctx, best)
    if use_cache:
        cache = _load()
        cache[key] = {"knobs": best, "ms": best_ms}
        _save(cache)
    return best, best_ms, table


def tune_hdc(ctx, X, Wt, reps=5, use_cache=True):
    """Pick the fastest HDC projection kernel (knob hdc_mode: persistent 128 x 256 tiles
    with 3 or 4 stages, in clusters of two sharing each W slice, 128 x 128 tiles, one
    tile per CTA) for this batch; a kernel the device refuses to launch is skipped."""
    B = X.shape[0]
    key = _key(ctx, ctx.groups(B)) + "|hdc|F%d|D%d" % (ctx.F, ctx.D)
    cache = _load() if use_cache else {}
    if use_cache and key in cache:
        apply(ctx, cache[key]["knobs"])
        return cache[key]["knobs"], cache[key]["ms"], []
    from .ephdc import EphdcError
    table = []
    for v in (0, 1, 2, 3, 4):
        try:
            ctx.tune_set("hdc_mode", v)
            ms = _time(lambda: ctx.hdc_encode(X, Wt), reps)
        except EphdcError:
            continue
        table.append((ms, {"hdc_mode": v}))
    if not table:
        raise RuntimeError("no HDC projection kernel could be launched")
    table.sort(key=lambda x: x[0])
    best_ms, best = table[0]
    apply(ctx, best)
    if use_cache:
        cache = _load()
        cache[key] = {"knobs": best, "ms": best_ms}
        _save(cache)
    return best, best_ms, table
