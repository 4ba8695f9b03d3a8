"""Measured pipe rates of the running GPU, per SM clock: the exp2 of the
special-function unit (the voxelizer's bound: one per in-box pair, Eq. 4) and
the FP32 FMA (its adjoint's bound), plain and packed.  The roofline peaks are
these rates x SMs x the SM clock sampled during the timed run.

    python -m paper_2411_04844_b300.peaks
"""
import json
import statistics

import torch

from . import dgr

KINDS = {"ex2": dgr.DGR_PIPE_EX2, "ffma": dgr.DGR_PIPE_FFMA, "ffma2": dgr.DGR_PIPE_FFMA2}


def pipe_rates(iters: int = 2048, blocks_per_sm: int = 4, repeats: int = 3) -> dict:
    """Operations per clock per SM for each pipe: per SM, the operations of
    its CTAs over (latest end - earliest start) in that SM's clock64; the
    median over SMs, best of `repeats` launches.  Also the SM count."""
    dev = torch.cuda.current_device()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    nb = sms * blocks_per_sm
    rec = torch.zeros(4 * nb, dtype=torch.int64, device="cuda")
    sink = torch.zeros(256 * nb, device="cuda")
    out = {"sms": sms}
    for name, kind in KINDS.items():
        dgr.dgr_pipe_rate(kind, 64, nb, rec, sink)  # warm-up (module load, clocks)
        best = 0.0
        for _ in range(repeats):
            dgr.dgr_pipe_rate(kind, iters, nb, rec, sink)
            r = rec.view(nb, 4).cpu().tolist()
            per_sm = {}
            for sm, t0, t1, ops in r:
                a = per_sm.setdefault(sm, [t0, t1, 0])
                a[0], a[1], a[2] = min(a[0], t0), max(a[1], t1), a[2] + ops
            rates = [ops / max(t1 - t0, 1) for t0, t1, ops in per_sm.values()]
            best = max(best, statistics.median(rates))
        out[name] = best
    return out


def l2_rates(mib: int = 48, passes: int = 20, blocks_per_sm: int = 8, repeats: int = 3) -> dict:
    """L2 bandwidth in GB/s over an L2-resident buffer of `mib` MiB: streaming
    reads and 32-bit integer reductions (best of `repeats`, CUDA events, the
    first pass after a warm-up pass that brings the buffer into L2)."""
    dev = torch.cuda.current_device()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    nb = sms * blocks_per_sm
    buf = torch.zeros(mib * 2 ** 20 // 4, device="cuda")
    sink = torch.zeros(256 * nb, device="cuda")
    out = {"buffer_mib": mib}
    for name, kind in (("read", 0), ("red_s32", 1)):
        dgr.dgr_l2_rate(kind, buf, 1, nb, sink)
        best = 0.0
        for _ in range(repeats):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            dgr.dgr_l2_rate(kind, buf, passes, nb, sink)
            e1.record()
            torch.cuda.synchronize()
            best = max(best, buf.numel() * 4.0 * passes / (e0.elapsed_time(e1) / 1e3) / 1e9)
        out[name + "_gbs"] = best
    return out


if __name__ == "__main__":
    print(json.dumps({**pipe_rates(), "l2": l2_rates()}))
