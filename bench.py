#!/usr/bin/env python
"""Benchmark: ms per conv2d + bootstrap block at N = 2^16 (config 2).

One step = one Alg. 1 block (fused CinS conv -> ModRaise -> CtoS -> EvalMod(Re, Im)
-> mask -> StoC1) on one ciphertext holding 16 channels of 32 x 32 (padded to 64 x 64),
with 3x3 Gaussian(0, 0.1) weights.  Keys, plaintext diagonals and the input
ciphertext are resident in HBM before the timed region; the working set (rotation
keys alone are several GB) is far larger than the 129 MB L2, so no flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle instead.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as WL  # noqa: E402

METRIC = "ms per conv2d+bootstrap block at N=2^16"
# DRAM bytes (read + write) per algorithmic byte of a forward NTT done as two k_ntt16 passes
# (one read and one write of the limbs per transform are the algorithmic bytes, 268.4 MB for 256
# limbs): ncu (--set full, one forward transform of 256 limbs at N = 2^16, cold caches) counted
# 134.4 + 81.0 MB for the first pass and 186.5 + 89.4 MB for the second; traffic of a launch
# scales with its limbs, so the in-block traffic per launch is this ratio times the launch's
# algorithmic bytes.
NTT_FWD_DRAM_PER_ALGO_BYTE = (134.4 + 81.0 + 186.5 + 89.4) / 268.4
# The same ratio at the block's own launch sizes (at most ~70 limbs, so the whole transform
# fits in the 129 MB L2): ncu with warm caches (no flush, as in the block) on a 24-limb forward
# transform counted 0.005 + 0.050 MB (first pass) and 0.082 + 0.025 MB (second pass) of DRAM
# traffic for 25.2 MB of algorithmic bytes.
NTT_FWD_DRAM_PER_ALGO_BYTE_IN_L2 = (0.005120 + 0.049920 + 0.082432 + 0.025088) / (2 * 24 * 0.524288)
L2_BYTES = 129e6
# The same ratio for the key-switch inner product, from an ncu capture (cold caches) of one
# launch at the top level (`--kernel ks`): 3 digits x 31 extended limbs with the automorphed c0
# term on 24 rows = (3*3 + 2) * 31 + 24 = 365 limbs of algorithmic traffic (191.4 MB); DRAM
# read 146.3 MB + write 3.6 MB.
KS_DRAM_PER_ALGO_BYTE = (146.3 + 3.6) / (365 * 65536 * 8 / 1e6)
ROOF_NOTES = {
    "ntt_fwd": "integer-multiply-pipe bound (fmaheavy 67-74% busy, DRAM 24-35% under ncu): the roofline is that "
               "pipe's (64 lanes per SM per clock, 16 lane-cycles per 64-bit Shoup butterfly); hbm_view gives "
               "the same launches against HBM",
    "bsgs_fused": "integer-multiply-pipe bound after asynchronous staging (fmaheavy 77% busy, DRAM 46% under ncu)",
    "ks_inner": "HBM bound: switching keys streamed once (evict-first), raised digits gathered through the Galois "
                "permutation; DRAM 55% of peak under ncu with cold caches",
}
CONFIG = "cfg2"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-small", action="store_true",
                    help="--impl reference: the config-2 chain at N=2^10 (checks the arm quickly; not a measurement)")
    ap.add_argument("--nvtx", action="store_true", help="mark the timed region with an NVTX range 'timed'")
    ap.add_argument("--batch", type=int, default=8, help="ciphertexts run concurrently for the batched figure")
    ap.add_argument("--workload", default="block", choices=["block", "ds", "serve", "batch", "cfg4", "serve5"],
                    help="block: the Alg. 1 block (default); ds: the downsampling layer of Alg. 2; "
                         "serve: the serving loop under Poisson arrivals; batch: 64 uneven-shape blocks "
                         "(ResNet-20 stage shapes) batched through the serving runtime; cfg4: ResNet-18-shaped "
                         "layers; serve5: whole ResNet-20 / ResNet-18-shaped requests through the serving loop")
    ap.add_argument("--batch-size", type=int, default=64, help="batch: number of seeded inputs")
    ap.add_argument("--serve-seconds", type=float, default=4.0, help="serve: seconds of arrivals per rate")
    ap.add_argument("--variant", type=int, default=-1, help="--kernel ntt: time one launch variant only")
    ap.add_argument("--ntt-choice", default=None,
                    help="comma list of 8 NTT variants per size class (as 'autotune' reports them): used "
                         "instead of timing the variants, e.g. to profile the configuration of a plain run")
    ap.add_argument("--bsgs-splits", default=None,
                    help="comma list of baby-step counts per bootstrapping level, used instead of tuning")
    ap.add_argument("--limbs", type=int, default=256, help="--kernel ntt: limbs per launch")
    ap.add_argument("--kernel", default=None, choices=["ntt", "ks", "bsgs", "bblock", "conv"],
                    help="time one kernel family alone on a buffer larger than L2 (for profiling)")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------ replicas (N > 1) -----
def rank_info():
    """(rank, world, local rank) from the launcher's environment (1 process when absent)"""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x, dist, device="cpu"):
    """the slowest replica's value (every rank gets it); x unchanged without a process group"""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_ms_per_block(t_ms_max, steps, world):
    """replicas: `world` ranks each ran `steps` blocks within t_ms_max (the slowest rank's time),
    so the whole job's ms per block is t_ms_max / (steps * world); per-step time is per rank"""
    return t_ms_max / steps, t_ms_max / (steps * world)


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "fallback": True}


# Integer-multiply roofline of the N = 2^16 NTT.  A 64-bit Shoup butterfly needs a 64x64 high
# product (four 32x32 -> 64 partial products) and two 64x64 low products (one 32x32 -> 64 and
# two 32x32 -> 32 each): 6 wide + 4 narrow 32-bit multiplies, 16 lane-cycles of the integer
# multiply (fmaheavy) pipe counting a wide product as two.  That pipe retires 16 lanes per
# SM sub-partition per clock, 64 per SM: peak butterflies/s = 64 * SMs * clock / 16.  A
# transform of one limb does 16 stages of N/2 butterflies and has 2 N 8 algorithmic bytes (one
# read, one write), so the butterflies are the algorithmic bytes / 2 (per pass or per launch).
NTT_MUL_LANE_CYCLES_PER_BUTTERFLY = 16
GB300_SMS = 152


def ntt_alu_roofline(kst, pk):
    mhz = pk.get("sm_max_mhz", 2070.0)
    peak = 64.0 * GB300_SMS * mhz * 1e6 / NTT_MUL_LANE_CYCLES_PER_BUTTERFLY / 1e9     # G butterflies/s
    out = {"bound": "alu", "pipe": "integer multiply (fmaheavy)", "unit": "Gbutterfly/s",
           "peak": round(peak, 1), "peak_source": "152 SMs x 64 multiply lanes x %.0f MHz / %d lane-cycles "
           "per 64-bit Shoup butterfly (derived)" % (mhz, NTT_MUL_LANE_CYCLES_PER_BUTTERFLY)}
    for k in ("ntt_fwd", "ntt_inv"):
        v = kst.get(k)
        if v:
            ach = v["bytes"] / 2.0 / (v["ms"] * 1e-3) / 1e9
            out[k] = {"achieved": round(ach, 1), "frac": round(ach / peak, 4)}
    return out


# ------------------------------------------------------------- workload -----
def block_setup(K, torch, seed=1, tune=False, ntt_choice=None, bsgs_splits=None):
    """context, conv plan, bootstrapping configuration, keys and one encrypted input of the
    config-2 block; with tune, the NTT launch variants and then the BSGS split of every
    bootstrapping level are autotuned before the keys are generated (or set from ntt_choice /
    bsgs_splits, comma lists, when given)"""
    d = WL.PARAMS[CONFIG]
    spec = WL.CONV[CONFIG]
    w = 1
    while w < spec["w0"] + spec["f"] // 2:
        w *= 2
    ctx = K.ckks_ctx_create(d, seed, torch.cuda.current_stream().cuda_stream)
    q, p, psi, delta = K.ckks_ctx_info(ctx)
    bt = K.ckks_boot_create(ctx, w, spec["w0"], spec["cout"])
    tuned = {}
    if tune:
        if ntt_choice:
            K.ckks_ctx_set_ntt_choices(ctx, [int(v) for v in ntt_choice.split(",")])
            tuned["ntt_variant_per_size_class"] = [int(v) for v in ntt_choice.split(",")]
            tuned["ntt_source"] = "given"
        else:
            tuned["ntt_variant_per_size_class"] = K.ckks_autotune(ctx, 3)
        tuned["bsgs_B_default"] = K.ckks_boot_bsgs_splits(bt)
        if bsgs_splits:
            K.ckks_boot_set_bsgs_splits(ctx, bt, [int(v) for v in bsgs_splits.split(",")])
            tuned["bsgs_B"] = K.ckks_boot_bsgs_splits(bt)
            tuned["bsgs_source"] = "given"
        else:
            tuned["bsgs_B"] = K.ckks_boot_tune_bsgs(ctx, bt, 3)
    delta0 = 2.0 ** 49
    x = WL.image(seed, spec["cin"], spec["w0"])
    W = WL.weights(seed, spec["cout"], spec["cin"], spec["f"], spec["weight"])
    conv = K.ckks_ptset_conv_fused(ctx, W, spec["cin"], spec["cout"], spec["f"], w, 1, (delta0 * q[1]) / delta[1])
    rots = sorted(set(K.ckks_ptset_rotations(conv)) | set(K.ckks_boot_rotations(bt)))
    keys = K.ckks_keygen(ctx, rots, True)
    ct = K.ckks_encrypt(ctx, keys, K.ckks_encode_image(ctx, x, w, 1, delta[1]), 1)
    K.ckks_sync(ctx)
    return dict(ctx=ctx, keys=keys, bt=bt, conv=conv, ct=ct, x=x, W=W, w=w, spec=spec, rots=rots, tuned=tuned)


def check_accuracy(K, s, out):
    """decoded block output vs the masked FP64 conv2d (max abs error)"""
    spec = s["spec"]
    got = K.ckks_decode_image(s["ctx"], K.ckks_decrypt(s["ctx"], s["keys"], out), spec["cout"], spec["w0"], s["w"])
    x, W = s["x"], s["W"]
    c = spec["f"] // 2
    h = spec["w0"]
    xp = np.zeros((x.shape[0], h + 2 * c, h + 2 * c))
    xp[:, c:c + h, c:c + h] = x
    ref = np.zeros((W.shape[0], h, h))
    for a in range(spec["f"]):
        for b in range(spec["f"]):
            ref += np.einsum("oi,ihw->ohw", W[:, :, a, b], xp[:, a:a + h, b:b + h])
    return float(np.abs(got - ref).max())


def lockstep_batches(K, torch, s, B, rounds, timing_B=0):
    """Config 3's batched figure: for each stride-1 block shape of the three stages of a
    ResNet-20-shaped network (16 x 32 x 32, 32 x 16 x 16, 64 x 8 x 8 channels x pixels; the first
    is the config-2 block), B seeded inputs run as ONE lockstep batch (ckks_block_batched,
    recorded as one CUDA graph: every kernel launched once for the B ciphertexts, keys and
    diagonals shared through L2), against the same block one ciphertext at a time (its own
    graph, replayed B times).  Every batched output equals the one-at-a-time output of its
    input; one output per shape is decoded against FP64 conv2d.  With timing_B, one eager batch
    of timing_B config-2 ciphertexts is timed per kernel (the batched rooflines)."""
    ctx, keys = s["ctx"], s["keys"]
    q, p, psi, delta = K.ckks_ctx_info(ctx)
    stream = torch.cuda.current_stream()
    out = {}
    kst = None
    for nm in ("cfg3_s1", "cfg3_s2", "cfg3_s3"):
        spec = WL.CONV[nm]
        w = 1
        while w < spec["w0"] + spec["f"] // 2:
            w *= 2
        if nm == "cfg3_s1":
            bt, conv, W = s["bt"], s["conv"], s["W"]
        else:
            bt = K.ckks_boot_create(ctx, w, spec["w0"], spec["cout"])
            W = WL.weights(11, spec["cout"], spec["cin"], spec["f"], spec["weight"])
            conv = K.ckks_ptset_conv_fused(ctx, W, spec["cin"], spec["cout"], spec["f"], w, 1,
                                           (2.0 ** 49 * q[1]) / delta[1])
            K.ckks_keys_add_rotations(ctx, keys, sorted(set(K.ckks_ptset_rotations(conv)) |
                                                        set(K.ckks_boot_rotations(bt))))
        xs = [WL.image(2000 + b, spec["cin"], spec["w0"]) for b in range(B)]
        ins = [K.ckks_encrypt(ctx, keys, K.ckks_encode_image(ctx, x, w, 1, delta[1]), 2000 + b)
               for b, x in enumerate(xs)]
        outs = [K.ckks_ct_create(ctx) for _ in range(B)]
        g = K.ckks_block_batched_graph_create(ctx, keys, ins, conv, bt, outs)
        one_out = K.ckks_ct_create(ctx)
        g1 = K.ckks_block_graph_create(ctx, keys, ins[0], conv, bt, one_out)
        K.ckks_graph_launch(g)
        K.ckks_graph_launch(g1)
        K.ckks_sync(ctx)

        def timed(fn):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)

        t_batch = timed(lambda: [K.ckks_graph_launch(g) for _ in range(rounds)]) / rounds
        t_one = timed(lambda: [K.ckks_graph_launch(g1) for _ in range(B)]) / B
        # every batched output against its input's own block (checked on up to 4 inputs)
        same = True
        for b in range(min(B, 4)):
            if b:
                K.ckks_ct_copy_into(ctx, ins[b], ins[0])
            K.ckks_graph_launch(g1)
            K.ckks_sync(ctx)
            same = same and bool((K.ckks_ct_export_rns(ctx, one_out) == K.ckks_ct_export_rns(ctx, outs[b])).all())
        got = K.ckks_decode_image(ctx, K.ckks_decrypt(ctx, keys, outs[1]), spec["cout"], spec["w0"], w)
        err = float(np.abs(got - conv2d_same(xs[1], W)).max())
        out[nm] = {"shape": "%dx%dx%d" % (spec["cin"], spec["w0"], spec["w0"]), "B": B,
                   "ct_per_s": round(B / (t_batch / 1e3), 2), "ms_per_ct": round(t_batch / B, 3),
                   "one_at_a_time_ms": round(t_one, 3), "speedup": round(t_one / (t_batch / B), 3),
                   "outputs_equal_one_at_a_time": same, "decoded_max_abs_err": err,
                   "launches_per_batch": K.ckks_graph_info(g), "launches_per_block": K.ckks_graph_info(g1)}
        del g, g1, outs, ins, one_out
        K.ckks_sync(ctx)
        if nm == "cfg3_s1" and timing_B:
            ins = [K.ckks_encrypt(ctx, keys, K.ckks_encode_image(ctx, xs[b % B], w, 1, delta[1]), 3000 + b)
                   for b in range(timing_B)]
            K.ckks_ctx_set_side_streams(ctx, 0)
            K.ckks_ctx_reset_counters(ctx)
            K.ckks_ctx_set_timing(ctx, 1)
            K.ckks_block_batched(ctx, keys, ins, conv, bt)
            K.ckks_ctx_set_timing(ctx, 0)
            K.ckks_ctx_set_side_streams(ctx, 1)
            kst = K.ckks_ctx_kernel_stats(ctx)
            del ins
            K.ckks_sync(ctx)
    # the stride-2 entries of stages 2 and 3 (Alg. 2 layers, 16 x 32 x 32 -> 32 x 16 x 16 and
    # 32 x 16 x 16 -> 64 x 8 x 8) as lockstep batches of B and one at a time; their inputs are
    # EvalMod outputs of a config-2 bootstrap (the level and scale every such layer receives)
    x0 = K.ckks_conv2d_cins(ctx, keys, s["ct"], s["conv"])
    re, im = K.ckks_bootstrap(ctx, keys, s["bt"], x0)
    for nm, (w_in, h_in, cin, cout) in (("entry_s1_s2", (64, 32, 16, 32)), ("entry_s2_s3", (32, 16, 32, 64))):
        b_in = K.ckks_boot_create(ctx, w_in, h_in, cin, stride=2)
        b_out = K.ckks_boot_create(ctx, w_in // 2, h_in // 2, cout)
        Wd = WL.weights(12, cout, cin, 3, "gauss")
        cs = [K.ckks_ptset_conv_fused_s2(ctx, Wd, cin, cout, 3, w_in, 0, 1, (2.0 ** 49 * q[1]) / delta[1])]
        K.ckks_keys_add_rotations(ctx, keys, sorted(set(K.ckks_boot_rotations(b_in)) | set(K.ckks_boot_rotations(b_out))
                                                    | set(K.ckks_ptset_rotations(cs[0]))))

        def batch_call():
            return K.ckks_downsample_layer_batched(ctx, keys, [[re]] * B, [[im]] * B, b_in, cs, b_out)

        def one_call():
            return K.ckks_downsample_layer(ctx, keys, [re], [im], b_in, cs, b_out)
        batch_call()
        one_call()
        t_b = timed(lambda: batch_call())
        t_1 = timed(lambda: one_call())
        out[nm] = {"B": B, "ms_per_ct": round(t_b / B, 3), "one_at_a_time_ms": round(t_1, 3),
                   "speedup": round(t_1 / (t_b / B), 3), "execution": "eager (not a graph)"}
        K.ckks_sync(ctx)
    # a ResNet-20-shaped inference: 9 blocks per stage, the first block of stages 2 and 3 the
    # stride-2 entry (HActivation excluded as in the config-2 block)
    per = {k: (out[k]["ms_per_ct"], out[k]["one_at_a_time_ms"]) for k in out}
    inf_b = 9 * per["cfg3_s1"][0] + per["entry_s1_s2"][0] + 8 * per["cfg3_s2"][0] + per["entry_s2_s3"][0] + \
        8 * per["cfg3_s3"][0]
    inf_1 = 9 * per["cfg3_s1"][1] + per["entry_s1_s2"][1] + 8 * per["cfg3_s2"][1] + per["entry_s2_s3"][1] + \
        8 * per["cfg3_s3"][1]
    out["resnet20_inference"] = {"batched_ms_per_inference": round(inf_b, 1), "one_at_a_time_ms": round(inf_1, 1),
                                 "batched_inferences_per_s": round(1e3 / inf_b, 3),
                                 "how": "9 x 16x32x32 block + stride-2 entry + 8 x 32x16x16 + stride-2 entry + 8 x "
                                        "64x8x8, per-ciphertext times of B-wide lockstep batches"}
    return out, kst


def conv2d_same(x, W):
    """FP64 conv2d, stride 1, zero padding f // 2 (cross-correlation), x (cin, h, h), W (cout, cin, f, f)"""
    f = W.shape[2]
    c = f // 2
    h = x.shape[1]
    xp = np.zeros((x.shape[0], h + 2 * c, h + 2 * c))
    xp[:, c:c + h, c:c + h] = x
    ref = np.zeros((W.shape[0], h, h))
    for a in range(f):
        for b in range(f):
            ref += np.einsum("oi,ihw->ohw", W[:, :, a, b], xp[:, a:a + h, b:b + h])
    return ref


# ------------------------------------------------------------ oracle arm -----
# BSGS splits of the oracle's block (CtoS levels, StoC1 levels): the splits the GPU tuner picks
# on GB300 for config 2.
ORACLE_SPLITS = ([16, 16, 32], [16, 16, 8])
# Share of the whole oracle block taken by its first two steps (the fused conv; ModRaise and
# the first CtoS HMatmul), from a full block timed step by step with `--impl reference` on the
# GB300 machine's host (16 cores); the CPU baseline of the GPU arm times those two steps and
# divides by this share.
ORACLE_SAMPLE_SHARE = 0.145       # (1329.6 + 7203.6) / 58763.6 ms, Neoverse-V2 x 16
_ORACLE = {}


def _oracle_block(full, name=CONFIG):
    """The oracle on the config-2 chain with the block's plans, keys and input, made once per
    process (keys and plaintexts are resident in the GPU arm's timed block too).  full: keys
    for every step of the block; else only for its first two steps.  name = "cfg2_small" runs
    the same chain at N = 2^10 (a quick check of the reference arm, not a measurement)."""
    key = (full, name)
    if key not in _ORACLE:
        from oracle import boot as BT
        from oracle import encoding as E
        from oracle import params as PP
        from oracle.scheme import Oracle
        d = WL.PARAMS[name]
        spec = WL.CONV[name]
        P = PP.Params(d["log_n"], d["n_q"], d["dnum"], d["q0_bits"], d["scale_bits"], d["p_bits"], h=d["h"],
                      sigma=d["sigma"], n_p=d["n_p"], boot_bits=d["boot_bits"], n_boot=d["n_boot"])
        o = Oracle(P, 1)
        w = E.pad_width(spec["w0"], spec["f"])
        x = WL.image(1, spec["cin"], spec["w0"])
        W = WL.weights(1, spec["cout"], spec["cin"], spec["f"], spec["weight"])
        splits = ORACLE_SPLITS if name == CONFIG else (None, None)
        cfg = BT.BootConfig(o, w, spec["w0"], spec["cout"], ctos_B=splits[0], stoc_B=splits[1])
        plan = o.conv_plan(W, spec["cin"], spec["cout"], spec["f"], w, 1, (cfg.delta0 * float(P.q[1])) / P.delta[1])
        m = P.n // 2
        if full:
            o.gen_relin_key()
            o.gen_conj_key()
            o.gen_rotation_keys(BT.block_rotations(o, plan, cfg))
        else:
            o.gen_rotation_keys(sorted(set(plan.rotations(m)) | set(cfg.ctos[0].rotations(m))))
        ct = o.encrypt(o.encode_pt(E.cins_input_slots(x, w, P.n), 1, P.delta[1]), 1)
        _ORACLE[key] = (o, BT.block_stages(o, plan, cfg), ct)
    return _ORACLE[key]


def _cores():
    from oracle import _clib
    return _clib.max_threads()            # threads of the oracle's OpenMP loops


def _host_model():
    """the host CPU's model name (lscpu), e.g. to state which cores timed the oracle"""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return None


def oracle_cfg1_e2e():
    """config 1 end to end on the oracle: encode -> encrypt -> fused CinS conv -> decrypt ->
    decode, ms (keys made beforehand)"""
    from oracle import encoding as E
    from oracle import params as PP
    from oracle.scheme import Oracle
    d = WL.PARAMS["cfg1"]
    spec = WL.CONV["cfg1"]
    P = PP.Params(d["log_n"], d["n_q"], d["dnum"], d["q0_bits"], d["scale_bits"], d["p_bits"], h=d["h"],
                  sigma=d["sigma"])
    x = WL.image(0, spec["cin"], spec["w0"])
    W = WL.weights(0, spec["cout"], spec["cin"], spec["f"], spec["weight"])
    w = E.pad_width(spec["w0"], spec["f"])
    o = Oracle(P, 3)
    plan = o.conv_plan(W, 1, 1, spec["f"], w, P.L, (P.delta[P.L - 1] * float(P.q[P.L])) / P.delta[P.L])
    o.gen_rotation_keys(plan.rotations(P.n // 2))
    t0 = time.perf_counter()
    ct = o.encrypt(o.encode_pt(E.cins_input_slots(x, w, P.n), P.L, P.delta[P.L]), 1)
    out = o.conv2d_cins(ct, plan)
    E.conv_output_from_coeffs(o.decode_coeffs(o.decrypt(out)), P.n // (w * w), w * w, 1, w, spec["w0"])
    return (time.perf_counter() - t0) * 1e3


def oracle_sample():
    """CPU baseline of the GPU arm: the first two steps of the oracle's config-2 block (the fused
    conv; ModRaise and the first CtoS HMatmul) timed at the oracle's thread count and scaled by
    their measured share of a whole block; the fused conv also on one thread; config 1 end to
    end."""
    from oracle import _clib
    o, stages, ct = _oracle_block(full=False)
    times = {}
    v = [ct]
    for name, step in stages[:2]:
        t0 = time.perf_counter()
        v = step(v)
        times[name] = time.perf_counter() - t0
    cores = _cores()
    _clib.set_threads(1)
    try:
        t0 = time.perf_counter()
        stages[0][1]([ct])
        conv_1t = time.perf_counter() - t0
    finally:
        _clib.set_threads(cores)
    e2e1 = oracle_cfg1_e2e()
    sample_s = sum(times.values())
    value = sample_s / ORACLE_SAMPLE_SHARE * 1e3
    return {"value": round(value, 1), "unit": "ms", "cores": cores, "kind": "oracle",
            "sample": "oracle at N=2^16 on the config-2 chain: the block's first two steps measured (fused conv "
                      "%.2f s, ModRaise + first CtoS HMatmul %.2f s), divided by their share %.3f of a whole "
                      "oracle block timed step by step (--impl reference)" % (
                          times["conv"], times["modraise_ctos0"], ORACLE_SAMPLE_SHARE),
            "one_thread": {"step": "fused conv", "s": round(conv_1t, 3), "speedup": round(conv_1t / times["conv"], 2)},
            "cfg1_e2e_ms": round(e2e1, 1), "host": _host_model()}


def run_reference(args):
    """The oracle's whole config-2 block, measured: its steps (fused conv; ModRaise + CtoS
    HMatmul; two more CtoS HMatmuls; conjugate split; EvalMod Re; EvalMod Im; masks + Re + i Im;
    three StoC1 HMatmuls) run one per bench step, in order, the block starting over after its
    last step; `value` = the sum over the steps of each step's mean measured time, i.e. ms per
    block, every step measured (warm-up steps fill in a step the timed ones did not reach)."""
    rank, _, _ = rank_info()
    if rank != 0:      # under torchrun rank 0 alone times the oracle; the others exit without work
        return
    small = getattr(args, "oracle_small", False)
    t_setup = time.perf_counter()
    o, stages, ct = _oracle_block(full=True, name="cfg2_small" if small else CONFIG)
    t_setup = time.perf_counter() - t_setup
    S = len(stages)
    per = {name: [] for name, _ in stages}
    warm = {name: [] for name, _ in stages}
    v = [ct]
    timed_s = 0.0
    n_run = max(args.warmup + args.steps, S)       # at least one whole block
    for i in range(n_run):
        name, step = stages[i % S]
        if i % S == 0:
            v = [ct]
        t0 = time.perf_counter()
        v = step(v)
        dt = time.perf_counter() - t0
        if i < args.warmup:
            warm[name].append(dt)
        elif i < args.warmup + args.steps:
            per[name].append(dt)
            timed_s += dt
        else:
            warm[name].append(dt)
    stage_ms = {}
    for name, _ in stages:
        xs = per[name] or warm[name]
        stage_ms[name] = 1e3 * sum(xs) / len(xs) if xs else None
    measured = all(x is not None for x in stage_ms.values())
    value = sum(stage_ms.values()) if measured else None
    cores = _cores()
    sample = ("the oracle's whole config-2 block (N=2^16, 24 limbs, BSGS splits %s / %s) measured step by step: "
              "%d steps per block, one per bench step, block restarted after its last step; value = sum of each "
              "step's mean time%s" % (ORACLE_SPLITS[0], ORACLE_SPLITS[1], S,
                                      "" if all(per[n] for n, _ in stages) else
                                      " (steps outside the timed region measured in the warm-up or after it)"))
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 1) if value else None, "unit": "ms",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(timed_s * 1e3 / max(1, args.steps), 1), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": ("config-2 block: 16x32x32 -> 16, 3x3 conv fused with StoC2, full bootstrap, "
                                    "N=2^16, 24 limbs") if not small else
                                   "config-2 chain at N=2^10 (check of the arm only, not a measurement)",
                       "l2": "working set > L2", "steps_per_block": S,
                       "setup_s": round(t_setup, 1)},
            "stage_ms": {k: round(x, 1) for k, x in stage_ms.items() if x is not None},
            "cpu_baseline": {"value": round(value, 1) if value else None, "unit": "ms", "cores": cores,
                             "kind": "oracle", "sample": sample, "host": _host_model()},
            "e2e": {"value": round(value, 1) if value else None, "unit": "ms", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- GPU arm -----
def run_ours(args):
    import torch
    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2312_04356_gb300 import build
    build.build()
    import paper_2312_04356_gb300.ckks as K

    stream = torch.cuda.Stream()          # graphs cannot be captured on the legacy default stream
    torch.cuda.set_stream(stream)
    s = block_setup(K, torch, seed=1 + rank, tune=True, ntt_choice=args.ntt_choice, bsgs_splits=args.bsgs_splits)
    ctx = s["ctx"]
    tuned = s["tuned"]
    out = K.ckks_ct_create(ctx)
    for _ in range(args.warmup):
        K.ckks_block(ctx, s["keys"], s["ct"], s["conv"], s["bt"], out)
    K.ckks_sync(ctx)
    err = check_accuracy(K, s, out)
    # operation counts of one block, and of the same block without the zero-mask shortcut
    K.ckks_ctx_reset_counters(ctx)
    K.ckks_block(ctx, s["keys"], s["ct"], s["conv"], s["bt"], out)
    K.ckks_sync(ctx)
    counts = K.ckks_ctx_counters(ctx)
    K.ckks_ctx_reset_counters(ctx)
    x0 = K.ckks_conv2d_cins(ctx, s["keys"], s["ct"], s["conv"])
    re, im = K.ckks_bootstrap(ctx, s["keys"], s["bt"], x0)
    K.ckks_stoc1(ctx, s["keys"], re, im, s["bt"])
    K.ckks_sync(ctx)
    counts_full = K.ckks_ctx_counters(ctx)
    del x0, re, im

    # the block as a CUDA graph (one eager run inside, then capture)
    gout = K.ckks_ct_create(ctx)
    graph = K.ckks_block_graph_create(ctx, s["keys"], s["ct"], s["conv"], s["bt"], gout)
    per_graph = K.ckks_graph_info(graph)
    for _ in range(args.warmup):
        K.ckks_graph_launch(graph)
    K.ckks_sync(ctx)
    err_graph = check_accuracy(K, s, gout)

    sampler = ClockSampler(local)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = K.ckks_ctx_counters(ctx)["launches"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if args.nvtx:
        torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    for _ in range(args.steps):
        K.ckks_graph_launch(graph)
    e1.record(stream)
    torch.cuda.synchronize()
    if args.nvtx:
        torch.cuda.nvtx.range_pop()
    if dist:
        dist.barrier()
    t_ms = e0.elapsed_time(e1)
    launches = K.ckks_ctx_counters(ctx)["launches"] - launches0
    t_ms = max_over_ranks(t_ms, dist, "cuda")
    ms_per_step, value = job_ms_per_block(t_ms, args.steps, world)

    # batched: B independent inputs, one graph each, on B streams at once
    B = max(1, args.batch)
    d = WL.PARAMS[CONFIG]
    q, p, psi, delta = K.ckks_ctx_info(ctx)
    ins, outs, graphs = [], [], []
    for b in range(B):
        xb = WL.image(100 + b, s["spec"]["cin"], s["spec"]["w0"])
        ins.append(K.ckks_encrypt(ctx, s["keys"], K.ckks_encode_image(ctx, xb, s["w"], 1, delta[1]), 100 + b))
        outs.append(K.ckks_ct_create(ctx))
        graphs.append(K.ckks_block_graph_create(ctx, s["keys"], ins[b], s["conv"], s["bt"], outs[b]))
    streams = [torch.cuda.Stream() for _ in range(B)]
    K.ckks_sync(ctx)

    def batched_round(k):
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for st in streams:
            st.wait_event(start)
        for _ in range(k):
            for b in range(B):
                K.ckks_graph_launch(graphs[b], streams[b].cuda_stream)
        for st in streams:
            ev = torch.cuda.Event()
            ev.record(st)
            stream.wait_event(ev)
        stop.record(stream)
        torch.cuda.synchronize()
        return start.elapsed_time(stop)

    batched_round(1)
    tb = batched_round(args.steps)
    clocks = sampler.stop()
    batched = {"B": B, "ct_per_s": round(B * args.steps / (tb / 1e3), 2),
               "ms_per_ct": round(tb / (B * args.steps), 3), "streams": B,
               "how": "B block graphs launched round-robin on B CUDA streams"}

    # end to end through the C ABI with host buffers: import (H2D + NTT) into a staging handle,
    # copy into the graph's input, replay, export (iNTT + D2H)
    host_in = torch.empty(K.ckks_ct_export_rns(ctx, s["ct"]).size, dtype=torch.int64, pin_memory=True).numpy()
    host_in[:] = K.ckks_ct_export_rns(ctx, s["ct"]).reshape(-1).view(np.int64)
    lev_in, sc_in = K.ckks_ct_info(s["ct"])
    lev_out, _ = K.ckks_ct_info(gout)
    host_out = torch.empty(2 * (lev_out + 1) * ctx.n, dtype=torch.int64, pin_memory=True).numpy()
    stage = K.ckks_ct_create(ctx)
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        K.ckks_ct_import_rns(ctx, host_in.view(np.uint64), lev_in, sc_in, stage)
        K.ckks_ct_copy_into(ctx, stage, s["ct"])
        K.ckks_graph_launch(graph)
        K.lib().ckks_ct_export_rns(ctx, gout, host_out.ctypes.data_as(K.ctypes.c_void_p))
    e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps

    # per-kernel CUDA-event timing of one more (eager) block: roofline of the dominant kernel;
    # side streams off so that each kernel is timed alone, not while sharing the GPU
    K.ckks_ctx_set_side_streams(ctx, 0)
    K.ckks_ctx_reset_counters(ctx)
    K.ckks_ctx_set_timing(ctx, 1)
    K.ckks_block(ctx, s["keys"], s["ct"], s["conv"], s["bt"], out)
    K.ckks_ctx_set_timing(ctx, 0)
    K.ckks_ctx_set_side_streams(ctx, 1)
    kst = K.ckks_ctx_kernel_stats(ctx)
    total = sum(v["ms"] for v in kst.values())
    top = max(kst.items(), key=lambda kv: kv[1]["ms"])
    pk = peaks()
    # the events around every launch cost time of their own: the same block recorded as a graph
    # with the side streams off runs the same kernels one after another without them; the
    # difference per launch is charged to the events (what remains includes the graph's own
    # launch gaps, so the net figures are still a lower bound on the kernels' rates)
    K.ckks_ctx_set_side_streams(ctx, 0)
    sout = K.ckks_ct_create(ctx)
    sgraph = K.ckks_block_graph_create(ctx, s["keys"], s["ct"], s["conv"], s["bt"], sout)
    K.ckks_ctx_set_side_streams(ctx, 1)
    for _ in range(2):
        K.ckks_graph_launch(sgraph)
    torch.cuda.synchronize()
    se0, se1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    se0.record(stream)
    for _ in range(5):
        K.ckks_graph_launch(sgraph)
    se1.record(stream)
    torch.cuda.synchronize()
    serial_ms = se0.elapsed_time(se1) / 5
    del sgraph
    n_launch = sum(v["launches"] for v in kst.values())
    event_us = max(0.0, (total - serial_ms) * 1e3 / max(n_launch, 1))
    achieved = top[1]["bytes"] / (top[1]["ms"] * 1e-3) / 1e9
    per_launch = top[1]["bytes"] / top[1]["launches"]
    ratio = {"ntt_fwd": NTT_FWD_DRAM_PER_ALGO_BYTE, "ks_inner": KS_DRAM_PER_ALGO_BYTE}.get(top[0])
    if top[0] == "ntt_fwd" and per_launch < L2_BYTES:      # the average launch's data stays in L2
        ratio = NTT_FWD_DRAM_PER_ALGO_BYTE_IN_L2
    traffic = round(ratio * per_launch) if ratio else None
    roof = {"kernel": top[0], "bound": "hbm", "achieved": round(achieved, 1), "peak": pk.get("hbm_gbs"),
            "unit": "GB/s", "frac": round(achieved / pk.get("hbm_gbs"), 4), "traffic": traffic,
            "algorithmic_bytes_per_launch": round(per_launch),
            "traffic_source": ("DRAM bytes per algorithmic byte of the kernel's ncu capture at a launch size "
                               "that fits in L2 (warm caches, as in the block) x this launch's algorithmic bytes"
                               if ratio == NTT_FWD_DRAM_PER_ALGO_BYTE_IN_L2 else
                               "DRAM bytes per algorithmic byte of the kernel's ncu capture x this launch's "
                               "algorithmic bytes") if ratio else None,
            "note": ROOF_NOTES.get(top[0]),
            "share": round(top[1]["ms"] / total, 4),
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if not pk.get("fallback") else "fallback",
            "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                            "GBps": round(v["bytes"] / max(v["ms"], 1e-9) / 1e6, 1)}
                        for k, v in sorted(kst.items(), key=lambda kv: -kv[1]["ms"])[:8]}}
    if top[0] in ("ntt_fwd", "ntt_inv"):
        # the NTT is bound by the integer multiply pipe: report that roofline, keep the HBM view
        alu = ntt_alu_roofline(kst, pk)
        hbm_view = {k: roof[k] for k in ("achieved", "peak", "unit", "frac", "peak_source")}
        roof.update({"bound": "alu", "achieved": alu[top[0]]["achieved"], "peak": alu["peak"],
                     "unit": alu["unit"], "frac": alu[top[0]]["frac"], "peak_source": alu["peak_source"],
                     "hbm_view": hbm_view})
        net = {k: dict(v, ms=max(1e-6, v["ms"] - v["launches"] * event_us * 1e-3)) for k, v in kst.items()}
        alu_net = ntt_alu_roofline(net, pk)
        roof["net_of_event_overhead"] = {
            "achieved": alu_net[top[0]]["achieved"], "frac": alu_net[top[0]]["frac"],
            "event_us_per_launch": round(event_us, 2), "serial_graph_ms": round(serial_ms, 3),
            "event_timed_sum_ms": round(total, 3),
            "how": "kernel time minus launches x (sum of event-timed kernels - the same block as a graph "
                   "with side streams off) / launches"}
    # key switching as % of HBM (the second roofline this bench reports): the hoisted rotations of
    # every HMatmul run inside the fused BSGS kernel (key switch + inner sums), the other key
    # switches (giant steps, relinearisations) in the inner-product kernel; both stream the
    # switching keys and gather the raised digits.  ModUp / ModDown conversions and NTTs are
    # reported above.
    roof_ks = None
    parts = {}
    for name in ("bsgs_fused", "ks_inner"):
        v = kst.get(name)
        if v:
            gbs = v["bytes"] / (v["ms"] * 1e-3) / 1e9
            parts[name] = {"achieved": round(gbs, 1), "frac": round(gbs / pk.get("hbm_gbs"), 4),
                           "launches": v["launches"], "share": round(v["ms"] / total, 4)}
    if parts:
        b = sum(kst[k]["bytes"] for k in parts)
        ms = sum(kst[k]["ms"] for k in parts)
        gbs = b / (ms * 1e-3) / 1e9
        roof_ks = {"kernel": "+".join(parts), "bound": "hbm", "achieved": round(gbs, 1), "peak": pk.get("hbm_gbs"),
                   "unit": "GB/s", "frac": round(gbs / pk.get("hbm_gbs"), 4), "parts": parts,
                   "note": ROOF_NOTES.get("bsgs_fused")}
    roof_alu = ntt_alu_roofline(kst, pk)
    roof_alu["net_of_event_overhead"] = {
        k: v for k, v in ntt_alu_roofline({k: dict(v, ms=max(1e-6, v["ms"] - v["launches"] * event_us * 1e-3))
                                           for k, v in kst.items()}, pk).items() if k in ("ntt_fwd", "ntt_inv")}
    # config 3's lockstep batches (B inputs per stride-1 stage shape, one graph each) and the
    # per-kernel rooflines of one eager lockstep batch of config-2 blocks
    lock, kst_b = lockstep_batches(K, torch, s, max(1, args.batch_size), max(1, min(args.steps, 2)),
                                   timing_B=max(1, args.batch_size))
    roof_b = {"B": max(1, args.batch_size), "ntt_alu": ntt_alu_roofline(kst_b, pk)}
    parts_b = {}
    for name in ("bsgs_fused", "ks_inner"):
        v = kst_b.get(name)
        if v:
            gbs = v["bytes"] / (v["ms"] * 1e-3) / 1e9
            parts_b[name] = {"achieved": round(gbs, 1), "frac": round(gbs / pk.get("hbm_gbs"), 4),
                             "launches": v["launches"], "ms": round(v["ms"], 3)}
    roof_b["keyswitch_hbm"] = parts_b
    roof_b["note"] = ("algorithmic bytes count each switching key and plaintext diagonal once per batch launch "
                      "(the batch's CTAs share them through L2) and every ciphertext's own words")
    roof_b["kernels"] = {k: {"launches": v["launches"], "ms": round(v["ms"], 3)}
                         for k, v in sorted(kst_b.items(), key=lambda kv: -kv[1]["ms"])[:8]}
    # the serving loop (config 5's continuous batching, config-2 requests): capacity and one
    # Poisson load at 0.8 of it with 8 slots, beside one slot (the unbatched plain path)
    cap, loads, plain, _ = serve_figures(K, s, 8, 2.0, loads=(0.8,), with_plain=True)
    serving = {"slots": 8, "mix": "70% one config-2 block, 30% two-block chains; host limbs in and out",
               "capacity_closed_loop": cap, "poisson_0.8": loads[0], "plain_one_slot": plain}
    try:
        activation = activation_figures(K, torch, ctx, s["keys"], stream, ms_per_step)
    except Exception as e:  # reported beside the block, never required
        activation = {"failed": str(e)}
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        try:
            cpu = oracle_sample()
        except Exception as e:  # the baseline is reported, never required
            cpu = {"value": None, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle", "sample": "failed: %s" % e}
    line = {"metric": METRIC, "value": round(value, 3), "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "config-2 block: 16x32x32 -> 16, 3x3 conv fused with StoC2, full bootstrap "
                                   "(CtoS 3 levels, EvalMod deg 59 + 3 double angles, StoC1 3 levels), "
                                   "N=2^16, 24 limbs", "batch": 1, "l2": "working set > L2 (keys ~GBs)",
                       "decoded_max_abs_err": err, "decoded_max_abs_err_graph": err_graph,
                       "execution": "CUDA graph replay of the block",
                       "parallelism": "replicas" if world > 1 else "single"},
            "clocks": clocks, "gpu_launches": launches, "launches_per_block": per_graph,
            "batched": batched, "batched_lockstep": lock, "roofline_batched": roof_b, "serving": serving,
            "activation": activation,
            "autotune": tuned,
            "e2e": {"value": round(e2e_ms, 3), "unit": "ms", "h2d_bytes_per_step": int(host_in.nbytes),
                    "d2h_bytes_per_step": int(host_out.nbytes)},
            "roofline": roof, "roofline_keyswitch": roof_ks, "roofline_ntt_alu": roof_alu, "op_counts": counts,
            "op_counts_without_zero_mask_skip": counts_full,
            "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def activation_figures(K, torch, ctx, keys, stream, block_ms, reps=5):
    """HActivation (Alg. 1's activation step) at N = 2^16 as the composite polynomial ReLU
    x (1 + s3(s2(s1(x)))) / 2 of degrees (15, 15, 27), timed with CUDA events on its own: its
    levels do not fit after the block's, so in a network it runs after a bootstrap of its own.
    The stages are Chebyshev least-squares fits (numpy) of tanh(5x), tanh(5x) and
    (1 + tanh(8x)) / 2: the time depends on the degrees only, and the decoded output is compared
    with the same composite evaluated in FP64.  block_ms is one GPU's time per block, so that
    block_plus_activation_ms is one ciphertext's latency through both."""
    from numpy.polynomial import chebyshev as CH
    nodes = np.cos(np.pi * (np.arange(4096) + 0.5) / 4096)

    def fit(f, deg, odd):
        c = CH.chebfit(nodes, f(nodes), deg)
        if odd:
            c[0::2] = 0.0
        return c
    stages = [fit(lambda x: np.tanh(5 * x), 15, True), fit(lambda x: np.tanh(5 * x), 15, True),
              fit(lambda x: (1 + np.tanh(8 * x)) / 2, 27, False)]
    q, _, _, delta = K.ckks_ctx_info(ctx)
    lev = len(q) - 1
    v = np.random.default_rng(77).uniform(-1.0, 1.0, ctx.n // 2)
    ct = K.ckks_encrypt(ctx, keys, K.ckks_encode(ctx, v, lev, delta[lev]), 77)
    out = K.ckks_eval_relu(ctx, keys, ct, stages)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        K.ckks_eval_relu(ctx, keys, ct, stages, out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    y = v
    for c in stages:
        y = CH.chebval(y, c)
    dec = K.ckks_decode(ctx, K.ckks_decrypt(ctx, keys, out)).real
    lev_out, _ = K.ckks_ct_info(out)
    return {"relu_ms": round(ms, 3), "degrees": [15, 15, 27], "from_level": lev, "to_level": lev_out,
            "decoded_max_abs_err_vs_fp64_composite": float(np.abs(dec - v * y).max()),
            "block_plus_activation_ms": round(block_ms + ms, 3),
            "how": "eager calls (no graph) on a fresh encryption at the top level, mean of %d" % reps,
            "note": "in a network the activation needs one more bootstrap (about one block) before it"}


def run_ds(args):
    """Alg. 2 at N = 2^16: two ciphertexts of 16 channels 32 x 32 (w = 64), each the EvalMod
    output of a config-2 block, -> stride-2 tail (masks, Re + i Im, decomposition, S_{l/4<-1})
    -> two decomposed 3x3 stride-2 convs -> one bootstrap -> tail: 64 channels 16 x 16 (w = 32)"""
    import torch
    from paper_2312_04356_gb300 import build
    build.build()
    import paper_2312_04356_gb300.ckks as K
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    s = block_setup(K, torch, seed=1)
    ctx, spec, w = s["ctx"], s["spec"], s["w"]
    K.ckks_autotune(ctx, 3)
    q, p, psi, delta = K.ckks_ctx_info(ctx)
    C, w0 = spec["cout"], spec["w0"]
    bt_in = K.ckks_boot_create(ctx, w, w0, C, stride=2)
    bt_out = K.ckks_boot_create(ctx, w // 2, w0 // 2, 4 * C)
    W2 = WL.weights(2, 4 * C, 2 * C, 3, "normal")
    # inputs: the EvalMod outputs of two config-2 blocks (images 1 and 2)
    xs, res, ims = [], [], []
    for t in range(2):
        x = WL.image(1 + t, spec["cin"], w0)
        xs.append(x)
        ct = K.ckks_encrypt(ctx, s["keys"], K.ckks_encode_image(ctx, x, w, 1, delta[1]), 1 + t)
        x0 = K.ckks_conv2d_cins(ctx, s["keys"], ct, s["conv"])
        re, im = K.ckks_bootstrap(ctx, s["keys"], s["bt"], x0)
        res.append(re)
        ims.append(im)
    lev_c = 1       # the tails' outputs are brought to level 1 at its canonical scale
    convs = [K.ckks_ptset_conv_fused_s2(ctx, W2, 2 * C, 4 * C, 3, w, t, lev_c, (2.0 ** 49 * q[1]) / delta[1])
             for t in range(2)]
    rots = sorted((set(K.ckks_boot_rotations(bt_in)) | set(K.ckks_boot_rotations(bt_out))
                   | set(K.ckks_ptset_rotations(convs[0])) | set(K.ckks_ptset_rotations(convs[1])))
                  - set(s["rots"]))
    K.ckks_keys_add_rotations(ctx, s["keys"], rots)
    out = K.ckks_ct_create(ctx)
    K.ckks_ctx_reset_counters(ctx)
    K.ckks_downsample_layer(ctx, s["keys"], res, ims, bt_in, convs, bt_out, out)
    K.ckks_sync(ctx)
    counts = K.ckks_ctx_counters(ctx)
    # FP64 reference: stride-2 conv of the two blocks' (masked) conv outputs
    c1 = [np.zeros((C, w0, w0)) for _ in range(2)]
    for t in range(2):
        xp = np.zeros((spec["cin"], w0 + 2, w0 + 2))
        xp[:, 1:1 + w0, 1:1 + w0] = xs[t]
        for a in range(3):
            for b in range(3):
                c1[t] += np.einsum("oi,ihw->ohw", s["W"][:, :, a, b], xp[:, a:a + w0, b:b + w0])
    x1 = np.concatenate(c1)
    xp = np.zeros((2 * C, w0 + 2, w0 + 2))
    xp[:, 1:1 + w0, 1:1 + w0] = x1
    ref = np.zeros((4 * C, w0 // 2, w0 // 2))
    for a in range(3):
        for b in range(3):
            ref += np.einsum("oi,ihw->ohw", W2[:, :, a, b], xp[:, a:a + w0:2, b:b + w0:2])
    got = K.ckks_decode_image(ctx, K.ckks_decrypt(ctx, s["keys"], out), 4 * C, w0 // 2, w // 2)
    err = float(np.abs(got - ref).max())
    gout = K.ckks_ct_create(ctx)
    graph = K.ckks_downsample_layer_graph_create(ctx, s["keys"], res, ims, bt_in, convs, bt_out, gout)
    per_graph = K.ckks_graph_info(graph)
    for _ in range(args.warmup):
        K.ckks_graph_launch(graph)
    K.ckks_sync(ctx)
    same = bool((K.ckks_ct_export_rns(ctx, gout) == K.ckks_ct_export_rns(ctx, out)).all())
    sampler = ClockSampler(0)
    sampler.start()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        K.ckks_graph_launch(graph)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    t_ms = e0.elapsed_time(e1) / args.steps
    # the same layer's share per stage: the two tails, then conv + bootstrap + tail
    K.ckks_ctx_set_timing(ctx, 1)
    K.ckks_ctx_reset_counters(ctx)
    K.ckks_downsample_layer(ctx, s["keys"], res, ims, bt_in, convs, bt_out, out)
    K.ckks_ctx_set_timing(ctx, 0)
    kst = K.ckks_ctx_kernel_stats(ctx)
    top = max(kst.items(), key=lambda kv: kv[1]["ms"])
    pk = peaks()
    achieved = top[1]["bytes"] / (top[1]["ms"] * 1e-3) / 1e9
    line = {"metric": "ms per downsampling layer (Alg. 2) at N=2^16", "value": round(t_ms, 3), "unit": "ms",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_ms, 3),
            "higher_is_better": False, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "2 x (16 ch 32x32, w=64) EvalMod outputs -> stride-2 tail -> 2 decomposed "
                                   "3x3 stride-2 convs (64 out) -> 1 bootstrap -> StoC1 at w=32",
                       "decoded_max_abs_err": err, "graph_equals_eager": same,
                       "execution": "CUDA graph replay of the layer", "l2": "working set > L2 (keys ~GBs)"},
            "clocks": clocks, "launches_per_layer": per_graph, "op_counts": counts,
            "roofline": {"kernel": top[0], "bound": "hbm", "achieved": round(achieved, 1),
                         "peak": pk.get("hbm_gbs"), "unit": "GB/s", "frac": round(achieved / pk.get("hbm_gbs"), 4),
                         "traffic": None},
            "cpu_baseline": None}
    print(json.dumps(line), flush=True)


def polyphase(x):
    """the four stride-2 phases of each channel of x (c, h, h), h even: image 4i + q + 2p is
    x[i, p::2, q::2] (how a client lays out the input of a stride-2 first layer)"""
    c, h, _ = x.shape
    out = np.zeros((4 * c, h // 2, h // 2))
    for i in range(c):
        for p in range(2):
            for q in range(2):
                out[4 * i + q + 2 * p] = x[i, p::2, q::2]
    return out


def conv2d_stride2(x, W):
    """FP64 cross-correlation, stride 2, zero padding f // 2"""
    return conv2d_same(x, W)[:, ::2, ::2]


def run_cfg4(args):
    """ImageNet-shaped ResNet-18 layers at N = 2^16 (config 4: 224 x 224 x 3 input, He-normal
    weights), each timed on the GPU and combined into seconds per inference:
      stem       7x7 stride-2 conv 224^2 x 3 -> 112^2 x 64: the client encodes the polyphase images
                 of each input channel (one channel per ciphertext at width 256), the decomposed
                 5x5 kernels (Alg. 2) run as a unit-stride conv over 3 input ciphertexts; 16 output
                 ciphertexts (4 channels each at w = 128), each conv + bootstrap (ckks_block_multi)
      pool       3x3 stride-2 average pooling (the downsampling depthwise conv of Alg. 2) 112^2 x 64
                 -> 56^2 x 64: 4 output ciphertexts, each from 4 stride-2 tails (ckks_downsample_layer)
      stage k    3x3 convs at 56^2 x 64 (4 ciphertexts in and out), 28^2 x 128 (2), 14^2 x 256 (1) and
                 7^2 x 512 (1), each output ciphertext a block matrix-vector product over the inputs
                 (Sec. 3.3.3) with its bootstrap; the stride-2 3x3 entry conv of stages 2-4 and its
                 1x1 stride-2 shortcut as Alg. 2 layers
    per inference = stem + pool + 4 stage-1 convs + for stages 2-4 (entry + shortcut + 3 convs).
    HActivation is excluded as in the config-2 block (each conv layer carries its bootstrap);
    the residual additions are elementwise and not timed.  Layers are timed one at a time on
    inputs of their own shape (encrypted seeded images; the Alg. 2 layers on EvalMod outputs of
    a config-2 bootstrap, which have the same level and scale); the conv layers are decoded
    against FP64 conv2d."""
    import torch
    from paper_2312_04356_gb300 import build
    build.build()
    import paper_2312_04356_gb300.ckks as K
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    s = block_setup(K, torch, seed=1)
    ctx, keys = s["ctx"], s["keys"]
    tuned = K.ckks_autotune(ctx, 3)
    q, p, psi, delta = K.ckks_ctx_info(ctx)
    s_pt = (2.0 ** 49 * q[1]) / delta[1]
    rng = np.random.default_rng(44)
    have = set(s["rots"])

    def need(*objs):
        r = set()
        for o in objs:
            r |= set(K.ckks_ptset_rotations(o) if isinstance(o, K.PtSet) else K.ckks_boot_rotations(o))
        new = sorted(r - have)
        if new:
            K.ckks_keys_add_rotations(ctx, keys, new)
            have.update(new)

    def he(cout, cin, f):
        return rng.normal(0.0, np.sqrt(2.0 / (cin * f * f)), (cout, cin, f, f))

    def enc(imgs, w):
        return K.ckks_encrypt(ctx, keys, K.ckks_encode_image(ctx, imgs, w, 1, delta[1]), int(rng.integers(1 << 30)))

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn()                                             # warm-up (lazy tables, pool)
        torch.cuda.synchronize()
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), r

    def err_of(out, ref, w, c):
        got = K.ckks_decode_image(ctx, K.ckks_decrypt(ctx, keys, out), c, ref.shape[1], w)
        return float(np.abs(got - ref[:c]).max())

    layers = {}
    # EvalMod outputs of a config-2 bootstrap: inputs of every Alg. 2 layer (same level and scale)
    x0 = K.ckks_conv2d_cins(ctx, keys, s["ct"], s["conv"])
    re, im = K.ckks_bootstrap(ctx, keys, s["bt"], x0)

    # ---- stem
    x = WL.image(7, 3, 224)
    W = he(64, 3, 7)
    pp = polyphase(x)
    bt = K.ckks_boot_create(ctx, 128, 112, 4)
    sets = [[K.ckks_ptset_conv_fused_s2(ctx, W[4 * j:4 * j + 4], 3, 4, 7, 256, t, 1, s_pt) for t in range(3)]
            for j in range(16)]
    need(bt, *sets[0])
    ins = [enc(pp[4 * t:4 * t + 4], 128) for t in range(3)]
    t_ms, outs = timed(lambda: [K.ckks_block_multi(ctx, keys, ins, sets[j], bt) for j in range(16)])
    layers["stem"] = {"ms": round(t_ms, 2), "ciphertexts_out": 16, "inputs_per_output": 3,
                      "decoded_max_abs_err": err_of(outs[0], conv2d_stride2(x, W[:4]), 128, 4)}
    del sets, ins, outs

    # ---- Alg. 2 layers: (name, n outputs, inputs per output, bt_in (w, w0, cout), bt_out (w, w0, cout), set maker)
    def ds_layer(name, n_out, n_in, bin_, bout, make_set):
        b_in = K.ckks_boot_create(ctx, bin_[0], bin_[1], bin_[2], stride=2)
        b_out = K.ckks_boot_create(ctx, bout[0], bout[1], bout[2])
        sets_ = [make_set(t) for t in range(n_in)]
        need(b_in, b_out, *sets_)
        t_ms_, _ = timed(lambda: [K.ckks_downsample_layer(ctx, keys, [re] * n_in, [im] * n_in, b_in, sets_, b_out)
                                  for _ in range(n_out)])
        layers[name] = {"ms": round(t_ms_, 2), "ciphertexts_out": n_out, "inputs_per_output": n_in}

    ds_layer("pool", 4, 4, (128, 112, 4), (64, 56, 16),
             lambda t: K.ckks_ptset_dwconv_fused_s2(ctx, np.full((16, 3, 3), 1.0 / 9.0), 128, t, 1, s_pt))

    # ---- stride-1 stage convs: (name, channels, image width, ciphertexts)
    def stage_conv(name, c, h, n):
        w = 1
        while w < h + 1:
            w *= 2
        C = c // n
        b = K.ckks_boot_create(ctx, w, h, C)
        Wc = he(c, c, 3)
        sets_ = [[K.ckks_ptset_conv_fused(ctx, Wc[C * j:C * j + C, C * i:C * i + C], C, C, 3, w, 1, s_pt)
                  for i in range(n)] for j in range(n)]
        need(b, *sets_[0])
        xs = rng.random((c, h, h))
        ins_ = [enc(xs[C * i:C * i + C], w) for i in range(n)]
        t_ms_, outs_ = timed(lambda: [K.ckks_block_multi(ctx, keys, ins_, sets_[j], b) for j in range(n)])
        layers[name] = {"ms": round(t_ms_, 2), "ciphertexts_out": n, "inputs_per_output": n,
                        "decoded_max_abs_err": err_of(outs_[0], conv2d_same(xs, Wc[:C]), w, C)}

    stage_conv("stage1_conv_56x56x64", 64, 56, 4)
    for (name, cin, cout, h_in, n_in, n_out) in (("stage2", 64, 128, 56, 4, 2), ("stage3", 128, 256, 28, 2, 1),
                                                  ("stage4", 256, 512, 14, 1, 1)):
        w_in = 1
        while w_in < h_in + 1:
            w_in *= 2
        Cin = cin // n_in
        cpo = cout // n_out
        for f, tag in ((3, "entry"), (1, "shortcut_1x1")):
            Wd = he(cout, cin, f)
            ds_layer("%s_%s" % (name, tag), n_out, n_in, (w_in, h_in, Cin), (w_in // 2, h_in // 2, cpo),
                     lambda t, Wd=Wd, f=f: K.ckks_ptset_conv_fused_s2(ctx, Wd[:cpo], cin, cpo, f, w_in, t, 1, s_pt))
        stage_conv("%s_conv_%dx%dx%d" % (name, h_in // 2, h_in // 2, cout), cout, h_in // 2, n_out)
    L = layers
    total = (L["stem"]["ms"] + L["pool"]["ms"] + 4 * L["stage1_conv_56x56x64"]["ms"] +
             sum(L["%s_entry" % k]["ms"] + L["%s_shortcut_1x1" % k]["ms"] + 3 * L[n]["ms"]
                 for k, n in (("stage2", "stage2_conv_28x28x128"), ("stage3", "stage3_conv_14x14x256"),
                              ("stage4", "stage4_conv_7x7x512"))))
    line = {"metric": "seconds per ResNet-18-shaped inference at N=2^16 (projected from timed layers)",
            "value": round(total / 1e3, 3), "unit": "s", "n_gpus": 1, "higher_is_better": False, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": "config 4: 224x224x3 input, 7x7/2 stem, 3x3/2 avg pool, stages 56^2x64, "
                                   "28^2x128, 14^2x256, 7^2x512 (4 convs each; stride-2 entries and 1x1 stride-2 "
                                   "shortcuts as Alg. 2 layers); He-normal weights, inputs U[0,1)",
                       "projection": "stem + pool + 4 x stage1 conv + sum over stages 2-4 of (entry + shortcut + "
                                     "3 x conv); HActivation excluded; eager calls timed with CUDA events",
                       "autotune_ntt_variant_per_size_class": tuned},
            "layers": layers, "rotation_keys": len(have)}
    print(json.dumps(line), flush=True)


def serve_figures(K, s, slots, seconds, loads=(0.5, 0.8, 0.95), with_plain=False):
    """The serving loop at N = 2^16 (config-2 blocks): 70% one-block requests and 30% two-block
    chains, inputs and outputs as host limbs; a saturating closed loop gives the capacity, then
    Poisson arrivals at the given fractions of it; with_plain, the same closed loop with one slot
    (the unbatched plain GPU path).  Returns (capacity, [per-load figures], plain, model info)."""
    ctx = s["ctx"]
    q, p, psi, delta = K.ckks_ctx_info(ctx)
    inputs = []
    for i in range(4):
        x = WL.image(200 + i, s["spec"]["cin"], s["spec"]["w0"])
        ct = K.ckks_encrypt(ctx, s["keys"], K.ckks_encode_image(ctx, x, s["w"], 1, delta[1]), 200 + i)
        inputs.append(K.ckks_ct_export_rns(ctx, ct))
    K.ckks_sync(ctx)
    g = np.random.default_rng(17)

    def make(n_slots):
        srv = K.ckks_server_create(ctx, s["keys"], n_slots, 0)
        A = K.ckks_server_add_model(srv, [s["conv"]], [s["bt"]])
        B = K.ckks_server_add_model(srv, [s["conv"], s["conv"]], [s["bt"], s["bt"]])
        K.ckks_server_start(srv)
        return srv, A, B

    def run(srv, A, B, n_slots, rate, secs, closed=False):
        K.ckks_server_reset_stats(srv)
        ids = []
        t0 = time.perf_counter()
        t_next = t0
        n_req = 0
        while True:
            now = time.perf_counter()
            if now - t0 > secs:
                break
            if closed or now >= t_next:
                model = A if g.random() < 0.7 else B
                ids.append(K.ckks_server_submit(srv, model, inputs[n_req % len(inputs)], 1, delta[1]))
                n_req += 1
                t_next += float(g.exponential(1.0 / rate)) if not closed else 0.0
                if closed and len(ids) >= 4 * n_slots:
                    K.ckks_server_wait(srv, ids[-3 * n_slots], 120)
            else:
                time.sleep(min(t_next - now, 0.001))
        for r in ids:
            K.ckks_server_wait(srv, r, 300)
        t_end = time.perf_counter()
        for r in ids:
            K.ckks_server_result(srv, r, ctx.n)
        st = K.ckks_server_stats(srv)
        return {"offered_per_s": None if closed else round(rate, 2), "requests": len(ids),
                "completed_per_s": round(st["completed"] / (t_end - t0), 2), "p50_ms": round(st["p50_ms"], 2),
                "p99_ms": round(st["p99_ms"], 2), "mean_ms": round(st["mean_ms"], 2),
                "max_in_flight": int(st["max_in_flight"]), "failed": int(st["failed"])}

    srv, A, B = make(slots)
    info = [K.ckks_server_model_info(srv, A), K.ckks_server_model_info(srv, B)]
    run(srv, A, B, slots, 10.0, 1.0)                                   # warm-up
    cap = run(srv, A, B, slots, None, seconds, closed=True)           # saturating closed loop
    per_load = [run(srv, A, B, slots, f * cap["completed_per_s"], seconds) for f in loads]
    srv.close()
    plain = None
    if with_plain:
        srv, A, B = make(1)
        run(srv, A, B, 1, 10.0, 0.5)
        plain = run(srv, A, B, 1, None, seconds, closed=True)
        srv.close()
    return cap, per_load, plain, info


def run_serve(args):
    """The serving loop at N = 2^16 under Poisson arrivals: 70% one-block requests (a config-2
    block) and 30% two-block chains, at three offered loads relative to the measured capacity;
    --batch slots, no HBM budget.  Reports completed requests/s, p50/p99/mean latency per load,
    beside the unbatched plain path (one slot)."""
    import torch
    from paper_2312_04356_gb300 import build
    build.build()
    import paper_2312_04356_gb300.ckks as K
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    s = block_setup(K, torch, seed=1)
    K.ckks_autotune(s["ctx"], 3)
    slots = max(1, args.batch)
    sampler = ClockSampler(0)
    sampler.start()
    cap, loads, plain, info = serve_figures(K, s, slots, args.serve_seconds, with_plain=True)
    clocks = sampler.stop()
    line = {"metric": "serving: completed requests/s and latency at N=2^16 (Poisson mix)",
            "value": cap["completed_per_s"], "unit": "requests/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": "u64", "data": "synthetic",
            "config": {"workload": "70% one config-2 block, 30% chains of two blocks; requests carry host "
                                   "coefficient limbs in and out (H2D, NTT, blocks, iNTT, D2H)",
                       "slots": slots, "hbm_budget": 0, "footprint_bytes": [i["footprint"] for i in info],
                       "kernels_per_request": [i["kernels"] for i in info]},
            "capacity_closed_loop": cap, "poisson": loads, "plain_one_slot": plain, "clocks": clocks}
    print(json.dumps(line), flush=True)


def run_batch(args):
    """Batched uneven-shape blocks at N = 2^16: the stride-1 conv2d + bootstrap blocks of the three
    stages of a ResNet-20-shaped network (16 x 32 x 32, 32 x 16 x 16 and 64 x 8 x 8 channels x
    pixels), B seeded inputs mixed over the three shapes, run through the serving runtime with
    --batch slots (each slot a stream replaying the shape's recorded block graph; inputs and
    outputs as host limbs).  The plain figure runs the same B requests one at a time (one
    slot).  Batched outputs must equal the one-at-a-time outputs bit for bit; one output per
    shape is decoded against the FP64 conv2d."""
    import torch
    from paper_2312_04356_gb300 import build
    build.build()
    import paper_2312_04356_gb300.ckks as K
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = K.ckks_ctx_create(WL.PARAMS[CONFIG], 1, stream.cuda_stream)
    tuned = K.ckks_autotune(ctx, 3)
    q, p, psi, delta = K.ckks_ctx_info(ctx)
    delta0 = 2.0 ** 49
    names = ["cfg3_s1", "cfg3_s2", "cfg3_s3"]
    shapes = []
    rots = set()
    for nm in names:
        spec = WL.CONV[nm]
        w = 1
        while w < spec["w0"] + spec["f"] // 2:
            w *= 2
        bt = K.ckks_boot_create(ctx, w, spec["w0"], spec["cout"])
        W = WL.weights(11, spec["cout"], spec["cin"], spec["f"], spec["weight"])
        conv = K.ckks_ptset_conv_fused(ctx, W, spec["cin"], spec["cout"], spec["f"], w, 1, (delta0 * q[1]) / delta[1])
        rots |= set(K.ckks_ptset_rotations(conv)) | set(K.ckks_boot_rotations(bt))
        shapes.append(dict(name=nm, spec=spec, w=w, bt=bt, W=W, conv=conv))
    keys = K.ckks_keygen(ctx, sorted(rots), True)
    nreq = max(1, args.batch_size)
    pick = np.random.default_rng(23).integers(0, len(shapes), size=nreq)
    reqs = []
    for i in range(nreq):
        sh = shapes[int(pick[i])]
        x = WL.image(1000 + i, sh["spec"]["cin"], sh["spec"]["w0"])
        ct = K.ckks_encrypt(ctx, keys, K.ckks_encode_image(ctx, x, sh["w"], 1, delta[1]), 1000 + i)
        reqs.append((int(pick[i]), x, K.ckks_ct_export_rns(ctx, ct)))
    K.ckks_sync(ctx)

    def serve_all(slots):
        srv = K.ckks_server_create(ctx, keys, slots, 0)
        models = [K.ckks_server_add_model(srv, [sh["conv"]], [sh["bt"]]) for sh in shapes]
        K.ckks_server_start(srv)
        for mi, m in enumerate(models):                     # warm-up: one request per shape
            r = next(x for x in reqs if x[0] == mi) if any(x[0] == mi for x in reqs) else None
            if r is not None:
                K.ckks_server_wait(srv, K.ckks_server_submit(srv, m, r[2], 1, delta[1]), 300)
        K.ckks_server_reset_stats(srv)
        t0 = time.perf_counter()
        ids = [K.ckks_server_submit(srv, models[si], limbs, 1, delta[1]) for si, _, limbs in reqs]
        for rid in ids:
            assert K.ckks_server_wait(srv, rid, 600) == K.CKKS_REQ_DONE
        dt = time.perf_counter() - t0
        outs = [K.ckks_server_result(srv, rid, ctx.n) for rid in ids]
        st = K.ckks_server_stats(srv)
        info = [K.ckks_server_model_info(srv, m) for m in models]
        srv.close()
        return dt, outs, st, info

    sampler = ClockSampler(0)
    sampler.start()
    dt_b, outs_b, st_b, info = serve_all(max(1, args.batch))
    dt_1, outs_1, st_1, _ = serve_all(1)
    clocks = sampler.stop()
    identical = all((a[0] == b[0]).all() for a, b in zip(outs_b, outs_1))
    errs = {}
    for si, sh in enumerate(shapes):
        k = next((i for i, r in enumerate(reqs) if r[0] == si), None)
        if k is None:
            continue
        limbs, lev, sc = outs_b[k]
        got = K.ckks_decode_image(ctx, K.ckks_decrypt(ctx, keys, K.ckks_ct_import_rns(ctx, limbs, lev, sc)),
                                  sh["spec"]["cout"], sh["spec"]["w0"], sh["w"])
        x = reqs[k][1]
        c = sh["spec"]["f"] // 2
        h = sh["spec"]["w0"]
        xp = np.zeros((x.shape[0], h + 2 * c, h + 2 * c))
        xp[:, c:c + h, c:c + h] = x
        ref = np.zeros((sh["W"].shape[0], h, h))
        for a in range(sh["spec"]["f"]):
            for b in range(sh["spec"]["f"]):
                ref += np.einsum("oi,ihw->ohw", sh["W"][:, :, a, b], xp[:, a:a + h, b:b + h])
        errs[sh["name"]] = float(np.abs(got - ref).max())
    counts = [int((pick == i).sum()) for i in range(len(shapes))]
    line = {"metric": "batched ct/s: uneven-shape conv2d+bootstrap blocks at N=2^16",
            "value": round(nreq / dt_b, 2), "unit": "ct/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": "u64", "data": "synthetic",
            "config": {"workload": "ResNet-20 stage shapes (stride-1 blocks): 16x32x32, 32x16x16, 64x8x8; "
                                   "3x3 conv fused with StoC2 + full bootstrap each; host limbs in and out",
                       "batch": nreq, "per_shape_count": dict(zip(names, counts)), "slots": max(1, args.batch),
                       "footprint_bytes": [i["footprint"] for i in info],
                       "kernels_per_block": [i["kernels"] for i in info]},
            "plain_one_at_a_time": {"value": round(nreq / dt_1, 2), "unit": "ct/s", "p50_ms": round(st_1["p50_ms"], 2)},
            "batched_latency": {"p50_ms": round(st_b["p50_ms"], 2), "p99_ms": round(st_b["p99_ms"], 2),
                                "max_in_flight": int(st_b["max_in_flight"])},
            "outputs_identical_batched_vs_alone": bool(identical), "decoded_max_abs_err": errs,
            "autotune_ntt_variant_per_size_class": tuned, "clocks": clocks}
    print(json.dumps(line), flush=True)


def run_kernel_ntt(args):
    """forward + inverse NTT of --limbs limbs (256: 128 MiB, > L2) cycling over the config-2 primes"""
    import torch
    from paper_2312_04356_gb300 import build
    build.build()
    import paper_2312_04356_gb300.ckks as K
    d = WL.PARAMS[CONFIG]
    ctx = K.ckks_ctx_create(d, 1, torch.cuda.current_stream().cuda_stream)
    q, p, _, _ = K.ckks_ctx_info(ctx)
    mods = q + p
    nl = max(1, args.limbs)
    ids = [i % len(mods) for i in range(nl)]
    x = WL.residues(1, [mods[i] for i in ids], ctx.n)
    dev = torch.from_numpy(x.view(np.int64)).cuda()
    res = {}
    ok = True
    for variant in ((0, 1, 2, 3, 4, 5) if args.variant < 0 else (args.variant,)):
        K.ckks_ctx_set_ntt_variant(ctx, variant)
        for _ in range(args.warmup):
            K.ckks_ntt_forward(ctx, dev.data_ptr(), nl, ids)
            K.ckks_ntt_inverse(ctx, dev.data_ptr(), nl, ids)
        torch.cuda.synchronize()
        K.ckks_ctx_reset_counters(ctx)
        K.ckks_ctx_set_timing(ctx, 1)
        for _ in range(args.steps):
            K.ckks_ntt_forward(ctx, dev.data_ptr(), nl, ids)
            K.ckks_ntt_inverse(ctx, dev.data_ptr(), nl, ids)
        K.ckks_ctx_set_timing(ctx, 0)
        st = K.ckks_ctx_kernel_stats(ctx)
        ok = ok and bool((dev.cpu().numpy().view(np.uint64) == x).all())
        res[variant] = {k: {"launches": v["launches"], "us_per_launch": round(1e3 * v["ms"] / v["launches"], 2),
                            "GBps": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1)} for k, v in st.items()}
        alu = ntt_alu_roofline(st, peaks())
        for k in ("ntt_fwd", "ntt_inv"):
            if k in res[variant] and k in alu:
                res[variant][k]["hbm_frac"] = round(res[variant][k]["GBps"] / peaks()["hbm_gbs"], 4)
                res[variant][k]["Gbutterfly_s"] = alu[k]["achieved"]
                res[variant][k]["alu_frac"] = alu[k]["frac"]
    print(json.dumps({"kernel": "ntt", "limbs": nl, "N": ctx.n, "roundtrip_exact": ok, "per_variant": res}))


def run_kernel_bblock(args):
    """one config-2 block as a lockstep batch of --batch-size ciphertexts, eager, side streams off,
    per-kernel timing (a case small enough for ncu captures of the batched key-switch kernels)"""
    import torch
    from paper_2312_04356_gb300 import build
    build.build()
    import paper_2312_04356_gb300.ckks as K
    s = block_setup(K, torch, seed=1)
    ctx = s["ctx"]
    q, p, _, delta = K.ckks_ctx_info(ctx)
    B = max(1, args.batch_size)
    ins = [K.ckks_encrypt(ctx, s["keys"], K.ckks_encode_image(ctx, s["x"], s["w"], 1, delta[1]), 10 + b)
           for b in range(B)]
    K.ckks_ctx_set_side_streams(ctx, 0)
    for _ in range(args.warmup):
        K.ckks_block_batched(ctx, s["keys"], ins, s["conv"], s["bt"])
    K.ckks_sync(ctx)
    K.ckks_ctx_reset_counters(ctx)
    K.ckks_ctx_set_timing(ctx, 1)
    for _ in range(args.steps):
        outs = K.ckks_block_batched(ctx, s["keys"], ins, s["conv"], s["bt"])
    K.ckks_ctx_set_timing(ctx, 0)
    st = K.ckks_ctx_kernel_stats(ctx)
    err = check_accuracy(K, s, outs[0])
    res = {k: {"launches": v["launches"], "ms_per_block": round(v["ms"] / args.steps, 3),
               "GBps": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1)}
           for k, v in sorted(st.items(), key=lambda kv: -kv[1]["ms"])}
    print(json.dumps({"kernel": "bblock", "B": B, "N": ctx.n, "decoded_max_abs_err": err, "per_kernel": res}))


def run_kernel_bsgs(args):
    """one top-level HMatmul shaped like a CtoS level of the config-2 bootstrap (63 diagonals
    at stride 1024, B = 16, level 23, diagonals over Q_23 u P with random residues): the fused
    baby-rotation / inner-sum kernel plus its giant steps; about 3 GB on the device"""
    import torch
    from paper_2312_04356_gb300 import build
    build.build()
    import paper_2312_04356_gb300.ckks as K
    d = WL.PARAMS[CONFIG]
    ctx = K.ckks_ctx_create(d, 1, torch.cuda.current_stream().cuda_stream)
    q, p, _, delta = K.ckks_ctx_info(ctx)
    L = len(q) - 1
    count, B, step = 63, 16, 1024
    ps = K.ckks_ptset_create(ctx, -31 * step, step, count, B, L, float(q[L]))
    mods = q + p
    rows = [mods[i] for i in range(L + 1)] + list(p)
    for i in range(count):
        K.ckks_ptset_set_rns(ctx, ps, i // B, i % B, WL.residues(100 + i, rows, ctx.n))
    keys = K.ckks_keygen(ctx, K.ckks_ptset_rotations(ps), False)
    ct = K.ckks_encrypt(ctx, keys, K.ckks_encode(ctx, WL.slots(1, ctx.n // 2, 0.5), L, delta[L]), 1)
    for _ in range(args.warmup):
        K.ckks_bsgs(ctx, keys, ct, ps)
    K.ckks_sync(ctx)
    K.ckks_ctx_reset_counters(ctx)
    K.ckks_ctx_set_timing(ctx, 1)
    for _ in range(args.steps):
        K.ckks_bsgs(ctx, keys, ct, ps)
    K.ckks_ctx_set_timing(ctx, 0)
    st = K.ckks_ctx_kernel_stats(ctx)
    res = {k: {"launches": v["launches"], "us_per_launch": round(1e3 * v["ms"] / v["launches"], 2),
               "GBps": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1)} for k, v in st.items()}
    print(json.dumps({"kernel": "bsgs", "level": L, "count": count, "B": B, "N": ctx.n, "per_kernel": res}))


def run_kernel_ks(args):
    """hoisted rotations of one config-2 ciphertext at the top level (ModUp, key-switch inner
    product, ModDown): per-kernel times of the key switch alone, a few hundred MB on the device"""
    import torch
    from paper_2312_04356_gb300 import build
    build.build()
    import paper_2312_04356_gb300.ckks as K
    d = WL.PARAMS[CONFIG]
    ctx = K.ckks_ctx_create(d, 1, torch.cuda.current_stream().cuda_stream)
    q, p, _, delta = K.ckks_ctx_info(ctx)
    L = len(q) - 1
    steps = [1, 2, 3, 4]
    keys = K.ckks_keygen(ctx, steps, False)
    ct = K.ckks_encrypt(ctx, keys, K.ckks_encode(ctx, WL.slots(1, ctx.n // 2, 0.5), L, delta[L]), 1)
    for _ in range(args.warmup):
        K.ckks_rotate_hoisted(ctx, keys, ct, steps)
    K.ckks_sync(ctx)
    K.ckks_ctx_reset_counters(ctx)
    K.ckks_ctx_set_timing(ctx, 1)
    for _ in range(args.steps):
        K.ckks_rotate_hoisted(ctx, keys, ct, steps)
    K.ckks_ctx_set_timing(ctx, 0)
    st = K.ckks_ctx_kernel_stats(ctx)
    res = {k: {"launches": v["launches"], "us_per_launch": round(1e3 * v["ms"] / v["launches"], 2),
               "GBps": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1)} for k, v in st.items()}
    print(json.dumps({"kernel": "keyswitch", "level": L, "rotations_per_step": len(steps), "N": ctx.n,
                      "per_kernel": res}))


def run_serve5(args):
    """Config 5: the serving loop at N = 2^16 with whole-network requests, 70% ResNet-20-shaped
    stacks on CIFAR-shaped input (27 conv-bootstrap layers: 9 per stage at 16x32x32, 32x16x16 and
    64x8x8, the first of stages 2 and 3 an Alg. 2 stride-2 entry fed by the EvalMod outputs of the
    layer before it) and 30% ResNet-18-shaped stacks on ImageNet-shaped input (the 7x7 stride-2
    stem over three client-encoded polyphase ciphertexts into 16, the 3x3 stride-2 average pool
    into 4, stage convs whose channels span 4 / 2 / 1 / 1 ciphertexts, stride-2 entries; the 1x1
    shortcut branches and the residual additions are not part of the chained model), each as one
    recorded request graph per slot.  A saturating closed loop gives the capacity, then Poisson
    arrivals at 0.5 / 0.8 / 0.95 of it, beside the same closed loop on one slot (the unbatched
    plain path).  HActivation excluded as in the config-2 block; synthetic weights and inputs."""
    import torch
    from paper_2312_04356_gb300 import build
    build.build()
    import paper_2312_04356_gb300.ckks as K
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = K.ckks_ctx_create(WL.PARAMS[CONFIG], 1, stream.cuda_stream)
    tuned = K.ckks_autotune(ctx, 3)
    q, p, psi, delta = K.ckks_ctx_info(ctx)
    s_pt = (2.0 ** 49 * q[1]) / delta[1]
    rng = np.random.default_rng(55)
    t_setup = time.perf_counter()

    def he(cout, cin, f):
        return rng.normal(0.0, np.sqrt(2.0 / (cin * f * f)), (cout, cin, f, f))

    def conv_sets(c, n, w):                   # [n][n] sets of a stage conv over n ciphertexts
        C = c // n
        Wc = he(c, c, 3)
        return [[K.ckks_ptset_conv_fused(ctx, Wc[C * j:C * j + C, C * i:C * i + C], C, C, 3, w, 1, s_pt)
                 for i in range(n)] for j in range(n)]

    def entry_sets(cin, cout, n_in, n_out, w_in, f=3):
        cpo = cout // n_out
        Wd = he(cout, cin, f)
        return [[K.ckks_ptset_conv_fused_s2(ctx, Wd[cpo * j:cpo * j + cpo], cin, cpo, f, w_in, t, 1, s_pt)
                 for t in range(n_in)] for j in range(n_out)]

    B, D = K.CKKS_LAYER_BLOCK, K.CKKS_LAYER_DOWNSAMPLE
    boots, sets = [], []

    def boot(*a, **kw):
        b = K.ckks_boot_create(ctx, *a, **kw)
        boots.append(b)
        return b

    # ---- ResNet-20-shaped stack (27 layers)
    r20 = []
    stages = ((16, 32, 64), (32, 16, 32), (64, 8, 16))    # channels, image width, slice width
    for si, (c, h, w) in enumerate(stages):
        bt = boot(w, h, c)
        cs = conv_sets(c, 1, w)
        sets.extend(p for row in cs for p in row)
        n_blocks = 9 if si == 0 else 8
        last = si == len(stages) - 1
        for b in range(n_blocks):
            pre_ds = not last and b == n_blocks - 1
            bt_b = boot(w, h, c, stride=2) if pre_ds else bt
            r20.append(dict(kind=B, convs=cs, boot=bt_b))
        if not last:
            c2, h2, w2 = stages[si + 1]
            es = entry_sets(c, c2, 1, 1, w)
            sets.extend(p for row in es for p in row)
            r20.append(dict(kind=D, convs=es, boot=boot(w2, h2, c2), boot_in=r20[-1]["boot"]))
    # ---- ResNet-18-shaped stack (18 layers)
    r18 = []
    W = he(64, 3, 7)
    stem = [[K.ckks_ptset_conv_fused_s2(ctx, W[4 * j:4 * j + 4], 3, 4, 7, 256, t, 1, s_pt) for t in range(3)]
            for j in range(16)]
    sets.extend(p for row in stem for p in row)
    bt_in = boot(128, 112, 4, stride=2)
    r18.append(dict(kind=B, convs=stem, boot=bt_in))
    pool = [K.ckks_ptset_dwconv_fused_s2(ctx, np.full((16, 3, 3), 1.0 / 9.0), 128, t, 1, s_pt) for t in range(4)]
    sets.extend(pool)
    r18.append(dict(kind=D, convs=[pool] * 4, boot=boot(64, 56, 16), boot_in=bt_in, n_in=16,
                    inputs=[[4 * j + t for t in range(4)] for j in range(4)]))
    shapes = ((64, 56, 64, 4), (128, 28, 32, 2), (256, 14, 16, 1), (512, 7, 8, 1))   # c, h, w, ciphertexts
    for si, (c, h, w, n) in enumerate(shapes):
        cs = conv_sets(c, n, w)
        sets.extend(p for row in cs for p in row)
        bt = boot(w, h, c // n)
        n_conv = 4 if si == 0 else 3
        last = si == len(shapes) - 1
        for b in range(n_conv):
            pre_ds = not last and b == n_conv - 1
            r18.append(dict(kind=B, convs=cs, boot=boot(w, h, c // n, stride=2) if pre_ds else bt))
        if not last:
            c2, h2, w2, n2 = shapes[si + 1]
            es = entry_sets(c, c2, n, n2, w)
            sets.extend(p for row in es for p in row)
            r18.append(dict(kind=D, convs=es, boot=boot(w2, h2, c2 // n2), boot_in=r18[-1]["boot"]))
    rots = set()
    for x in sets:
        rots |= set(K.ckks_ptset_rotations(x))
    for b in boots:
        rots |= set(K.ckks_boot_rotations(b))
    keys = K.ckks_keygen(ctx, sorted(rots), True)
    # inputs: one 16 x 32 x 32 ciphertext; three polyphase ciphertexts of a 3 x 224 x 224 image
    x20 = K.ckks_ct_export_rns(ctx, K.ckks_encrypt(ctx, keys, K.ckks_encode_image(
        ctx, WL.image(301, 16, 32), 64, 1, delta[1]), 301))
    pp = polyphase(WL.image(302, 3, 224))
    x18 = np.stack([K.ckks_ct_export_rns(ctx, K.ckks_encrypt(ctx, keys, K.ckks_encode_image(
        ctx, pp[4 * t:4 * t + 4], 128, 1, delta[1]), 303 + t)) for t in range(3)])
    K.ckks_sync(ctx)
    setup_s = time.perf_counter() - t_setup
    g = np.random.default_rng(19)

    def make(n_slots):
        t0 = time.perf_counter()
        srv = K.ckks_server_create(ctx, keys, n_slots, 0)
        a = K.ckks_server_add_model_layers(srv, r20)
        b = K.ckks_server_add_model_layers(srv, r18)
        K.ckks_server_start(srv)
        return srv, a, b, time.perf_counter() - t0

    def run(srv, a, b, rate, secs, closed=False, n_slots=1):
        out_a, out_b = K.ckks_server_model_shape(srv, a)[1], K.ckks_server_model_shape(srv, b)[1]
        K.ckks_server_reset_stats(srv)
        ids = []
        t0 = time.perf_counter()
        t_next = t0
        while time.perf_counter() - t0 <= secs:
            now = time.perf_counter()
            if closed or now >= t_next:
                if g.random() < 0.7:
                    ids.append((K.ckks_server_submit(srv, a, x20, 1, delta[1]), out_a))
                else:
                    ids.append((K.ckks_server_submit(srv, b, x18, 1, delta[1]), out_b))
                t_next += 0.0 if closed else float(g.exponential(1.0 / rate))
                if closed and len(ids) >= 2 * n_slots:
                    K.ckks_server_wait(srv, ids[-2 * n_slots + 1][0], 600)
            else:
                time.sleep(min(t_next - now, 0.005))
        for r, _ in ids:
            K.ckks_server_wait(srv, r, 600)
        t_end = time.perf_counter()
        for r, n_out in ids:
            K.ckks_server_result(srv, r, ctx.n, n_out)
        st = K.ckks_server_stats(srv)
        return {"offered_per_s": None if closed else round(rate, 3), "requests": len(ids),
                "completed_per_s": round(st["completed"] / (t_end - t0), 3), "p50_ms": round(st["p50_ms"], 1),
                "p99_ms": round(st["p99_ms"], 1), "mean_ms": round(st["mean_ms"], 1),
                "max_in_flight": int(st["max_in_flight"]), "failed": int(st["failed"])}

    slots = max(1, args.batch)
    secs = max(4.0, float(args.serve_seconds))
    srv, a, b, rec_s = make(slots)
    info = {"resnet20": K.ckks_server_model_info(srv, a), "resnet18": K.ckks_server_model_info(srv, b),
            "resnet18_shape": K.ckks_server_model_shape(srv, b)}
    run(srv, a, b, 1.0, 2.0)                                               # warm-up
    cap = run(srv, a, b, None, secs, closed=True, n_slots=slots)
    loads = [run(srv, a, b, f * cap["completed_per_s"], secs) for f in (0.5, 0.8, 0.95)]
    srv.close()
    srv, a, b, _ = make(1)
    run(srv, a, b, 1.0, 1.0)
    plain = run(srv, a, b, None, secs, closed=True, n_slots=1)
    srv.close()
    line = {"metric": "requests/s of whole-network inference requests at N=2^16 (config 5 mix)",
            "value": cap["completed_per_s"], "unit": "requests/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": "u64", "data": "synthetic",
            "config": {"workload": "config 5: 70% ResNet-20-shaped stacks (27 layers), 30% ResNet-18-shaped stacks "
                                   "(18 layers, shortcut branches not chained); Poisson arrivals",
                       "slots": slots, "seconds_per_load": secs, "rotation_keys": len(rots),
                       "autotune_ntt_variant_per_size_class": tuned},
            "capacity_closed_loop": cap, "poisson": dict(zip(("0.5", "0.8", "0.95"), loads)),
            "plain_one_slot": plain, "models": info, "setup_s": round(setup_s, 1), "record_s": round(rec_s, 1)}
    print(json.dumps(line), flush=True)


def run_kernel_conv(args):
    """base conversion alone, on the tensor cores and on the integer pipe: the ModUp of one
    config-2 ciphertext at the top level (three digits of 8 limbs, 23 outputs each) and the
    ModDowns of four hoisted rotations (two polynomials, 7 -> 24 limbs), timed per kernel"""
    import torch
    from paper_2312_04356_gb300 import build
    build.build()
    import paper_2312_04356_gb300.ckks as K
    d = WL.PARAMS[CONFIG]
    ctx = K.ckks_ctx_create(d, 1, torch.cuda.current_stream().cuda_stream)
    q, p, _, delta = K.ckks_ctx_info(ctx)
    L = len(q) - 1
    steps = [1, 2, 3, 4]
    keys = K.ckks_keygen(ctx, steps, False)
    ct = K.ckks_encrypt(ctx, keys, K.ckks_encode(ctx, WL.slots(1, ctx.n // 2, 0.5), L, delta[L]), 1)
    out = {}
    for name, tc in (("tensor_1_thread_per_row", 1), ("tensor_2_threads_per_row", 2), ("integer", 0)):
        K.ckks_ctx_set_tensor_conversion(ctx, tc)
        for _ in range(args.warmup):
            K.ckks_rotate_hoisted(ctx, keys, ct, steps)
        K.ckks_sync(ctx)
        K.ckks_ctx_reset_counters(ctx)
        K.ckks_ctx_set_timing(ctx, 1)
        for _ in range(args.steps):
            K.ckks_rotate_hoisted(ctx, keys, ct, steps)
        K.ckks_ctx_set_timing(ctx, 0)
        v = K.ckks_ctx_kernel_stats(ctx)["base_convert"]
        out[name] = {"launches": v["launches"], "us_per_launch": round(1e3 * v["ms"] / v["launches"], 2),
                     "GBps": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1)}
    K.ckks_ctx_set_tensor_conversion(ctx, 1)
    print(json.dumps({"kernel": "base_convert", "level": L, "N": ctx.n, "rotations_per_step": len(steps),
                      "device_faults": K.ckks_ctx_take_device_faults(ctx), "per_kernel": out}))


if __name__ == "__main__":
    a = parse_args()
    if a.kernel == "conv":
        run_kernel_conv(a)
    elif a.kernel == "ntt":
        run_kernel_ntt(a)
    elif a.kernel == "ks":
        run_kernel_ks(a)
    elif a.kernel == "bsgs":
        run_kernel_bsgs(a)
    elif a.kernel == "bblock":
        run_kernel_bblock(a)
    elif a.workload == "ds" and a.impl == "ours":
        run_ds(a)
    elif a.workload == "serve" and a.impl == "ours":
        run_serve(a)
    elif a.workload == "batch" and a.impl == "ours":
        run_batch(a)
    elif a.workload == "cfg4" and a.impl == "ours":
        run_cfg4(a)
    elif a.workload == "serve5" and a.impl == "ours":
        run_serve5(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
