"""Benchmark: active-set local-optimisation iterations per second.

Workload: a 1,000,000-Gaussian clustered room scene (20 clusters, sigma 0.3,
[-5,5]^3), SH degree 3, four 1920x1080 views at 0, pi/2, pi, 3pi/2 on a ring of
radius 4, a change box around the cluster nearest view 0's image centre
holding 5% of the Gaussians, its Gaussians perturbed by N(0, 0.05) to make the
target scene; the active set comes from change-mask lifting (majority vote).
A step is one iteration of the hot path over all four views: project_and_bin
(active Gaussians re-projected, static ones cached per update), sort_keys,
render_forward with the fused L1 loss, render_backward, adam_step_active.

Prints one JSON line (rank 0). With --impl reference the CPU oracle is timed
instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "active-set iters/s (fwd+bwd+Adam) @1M Gaussians 1080p"
UNIT = "iters/s"
WORKLOAD = "1M-Gaussian clustered room, SH3, 4 views 1920x1080, 5% change box, L1"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=1_000_000)
    p.add_argument("--fraction", type=float, default=0.05)
    p.add_argument("--width", type=int, default=1920)
    p.add_argument("--height", type=int, default=1080)
    p.add_argument("--views", type=int, default=4)
    p.add_argument("--loss", default="l1", choices=["l1", "l1+ssim"],
                   help="l1+ssim: the base optimiser's (1 - 0.2) L1 + 0.2 D-SSIM")
    p.add_argument("--e2e-updates", type=int, default=5)
    p.add_argument("--iters-per-update", type=int, default=10)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-configs", action="store_true",
                   help="time the CPU oracle and the float32 CPU baseline on the plain, "
                        "local-update and FD workloads in full (no GPU needed) and exit")
    p.add_argument("--no-configs", action="store_true",
                   help="skip the other workloads (plain, local update, FD) and the 1/10%% sweep")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--serving-scenes", type=int, default=64)
    p.add_argument("--serving-seconds", type=float, default=30.0,
                   help="length of the Poisson stream at --serving-rate")
    p.add_argument("--serving-load-seconds", type=float, default=10.0,
                   help="length of the streams at 50%% and 90%% of the batched saturation rate")
    p.add_argument("--serving-rate", type=float, default=200.0)
    p.add_argument("--serving-slots", type=int, default=8)
    p.add_argument("--profile-iteration", action="store_true",
                   help="after the warm-up, run one eager iteration inside the NVTX range "
                        "'cls_iteration' (for ncu --nvtx-include) and exit")
    return p.parse_args()


# ---------------------------------------------------------------- helpers ---

class Clocks:
    """nvidia-smi sampled every 50 ms; only samples taken inside a timed
    window count (the nearest ones are used if the window is shorter than
    the sampling period, and flagged)."""

    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self, t0: float, t1: float):
        """Stop sampling; returns the summary of [t0, t1]."""
        import datetime as dt
        self.rows = []
        if self.p is None:
            return self.window(t0, t1)
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                ts = dt.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                self.rows.append((ts, float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.f.name)
        return self.window(t0, t1)

    def window(self, t0: float, t1: float):
        """Median SM clock, maximum clock and active throttle reasons of the
        samples taken inside [t0, t1] (the two nearest ones, flagged, if the
        window is shorter than the sampling period)."""
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = self.rows
        inside = [r for r in rows if t0 <= r[0] <= t1]
        flag = None
        if not inside and rows:
            mid = 0.5 * (t0 + t1)
            inside = sorted(rows, key=lambda r: abs(r[0] - mid))[:2]
            flag = "timed window shorter than the sampling period: nearest samples"
        reasons = set()
        for r in inside:
            for nm, val in zip(self.NAMES, r[3]):
                if val.lower() == "active":
                    reasons.add(nm)
        out = {"sm_mhz": statistics.median([r[1] for r in inside]) if inside else None,
               "sm_max_mhz": inside[0][2] if inside else None, "reasons": sorted(reasons),
               "samples": len(inside)}
        if flag:
            out["note"] = flag
        return out


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured", float(d.get("sm_max_mhz", 2070.0))
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback", 2070.0


# ALU peak of the FP32 pipes: 152 SMs x 128 FP32 lanes x 2 FLOP per FMA x clock.
def fp32_peak_tflops(sm_mhz: float, sms: int = 152) -> float:
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


# Algorithmic FP32 work per (pixel, list entry) evaluation: offsets (2), exponent
# (9), exp (1), alpha and clamp (2), then forward: transmittance test (2), weight
# (1), colour (6) = 21; backward (static entry): 1 - alpha and T recovery (2),
# weight (1), colour behind (6) = 23 (an active entry adds 32 for its gradient).
FWD_FLOP_PER_EVAL = 21
BWD_FLOP_PER_EVAL = 23


def walked_evaluations(bt):
    """(pixel, list entry) evaluations the render kernels actually perform in
    one pass, from the pass's own buffers: per pixel of a rendered tile that
    did not stop inside the tile's cached static prefix, the forward walks
    from the prefix end to its last contributor and the backward from the
    prefix end to min(last contributor, the tile's last active entry + 1).
    Also the full-list count (every pixel from position 0), for context."""
    import torch
    dev = bt.n_contrib.device
    T = bt.info.total_tiles
    tile_of = torch.empty(bt.info.total_pixels, dtype=torch.int64, device=dev)
    for j in range(bt.n_views):
        v = bt.view_tab[j]
        W, H = int(v.cam.width), int(v.cam.height)
        ys = torch.arange(H, device=dev).view(H, 1) // 16
        xs = torch.arange(W, device=dev).view(1, W) // 16
        tile_of[int(v.pix_base): int(v.pix_base) + W * H] = (
            int(v.tile_base) + ys * int(v.tiles_x) + xs).reshape(-1)
    rendered = torch.zeros(T, dtype=torch.bool, device=dev)
    nt = int(bt.n_active_tiles.item())
    rendered[bt.active_tiles[:nt].long()] = True
    tc = bt.tile_cache.view(T, 4).long()
    n_prefix = tc[:, 1]
    start = torch.where(n_prefix == -1, torch.zeros_like(n_prefix), n_prefix)
    last_active = tc[:, 3]
    on = rendered[tile_of]
    nc = bt.n_contrib.long()
    if bt.prefix_mode:
        done = bt.prefix_state.view(-1, 4)[:, 0] < 0
    else:
        done = torch.zeros_like(on)
    live = on & ~done
    st = start[tile_of]
    fwd = torch.clamp(nc - st, min=0)
    bwd = torch.clamp(torch.minimum(nc, last_active[tile_of] + 1) - st, min=0)
    return {"forward": int(fwd[live].sum().item()), "backward": int(bwd[live].sum().item()),
            "full_list": int(nc[on].sum().item())}


def _tile_maps(bt):
    """Per pixel its global tile id; per rendered tile whether it is listed."""
    import torch
    dev = bt.n_contrib.device
    tile_of = torch.empty(bt.info.total_pixels, dtype=torch.int64, device=dev)
    for j in range(bt.n_views):
        v = bt.view_tab[j]
        W, H = int(v.cam.width), int(v.cam.height)
        ys = torch.arange(H, device=dev).view(H, 1) // 16
        xs = torch.arange(W, device=dev).view(1, W) // 16
        tile_of[int(v.pix_base): int(v.pix_base) + W * H] = (
            int(v.tile_base) + ys * int(v.tiles_x) + xs).reshape(-1)
    return tile_of


def pair_producing_records(bt):
    """Records whose tile rectangle holds at least one rendered tile (they are
    counted, stamped and walked by the emission), from the records' centres
    and radii and a summed-area table of the tile mask per view."""
    import torch
    rec = bt.records.view(-1, 12)
    rad = rec[:, 11].contiguous().view(torch.int32).to(torch.float32)
    total = 0
    for j in range(bt.n_views):
        v = bt.view_tab[j]
        tx, ty = int(v.tiles_x), int(v.tiles_y)
        r = rec[int(v.rec_base): int(v.rec_base) + bt.scenes[v.scene].n]
        rj = rad[int(v.rec_base): int(v.rec_base) + bt.scenes[v.scene].n]
        on = (bt.tile_active[int(v.tile_base): int(v.tile_base) + tx * ty] > 0).view(ty, tx)
        sat = torch.zeros(ty + 1, tx + 1, dtype=torch.int64, device=on.device)
        sat[1:, 1:] = on.long().cumsum(0).cumsum(1)
        x0 = torch.floor((r[:, 0] - rj) / 16).clamp(0, tx - 1).long()
        x1 = torch.floor((r[:, 0] + rj) / 16).clamp(0, tx - 1).long()
        y0 = torch.floor((r[:, 1] - rj) / 16).clamp(0, ty - 1).long()
        y1 = torch.floor((r[:, 1] + rj) / 16).clamp(0, ty - 1).long()
        cnt = sat[y1 + 1, x1 + 1] - sat[y0, x1 + 1] - sat[y1 + 1, x0] + sat[y0, x0]
        total += int(((rj > 0) & (cnt > 0)).sum().item())
    return total


def walk_counts(bt):
    """Per pass, from its buffers: the list entries the forward pass needs
    per rendered tile (from the walk start, 0 or the cached prefix end, to the
    deepest pixel's last contributor; pixels that stopped inside the prefix do
    not walk), those the backward needs (to min(last contributor, the tile's
    last active entry + 1)), the pixels each walks, and (bucketed layout) the
    keys in the depth bins the forward sorts: from the bin holding the walk
    start to the bin holding its last entry, with those in bins above the
    renderer's own sort limit counted apart."""
    import torch
    nt = int(bt.n_active_tiles.item())
    tiles = bt.active_tiles[:nt].long()
    T = bt.info.total_tiles
    tile_of = _tile_maps(bt)
    tc = bt.tile_cache.view(T, 4).long()
    start_t = torch.where(tc[:, 1] == -1, torch.zeros_like(tc[:, 1]), tc[:, 1])
    rendered = torch.zeros(T, dtype=torch.bool, device=tiles.device)
    rendered[tiles] = True
    on = rendered[tile_of]
    done = bt.prefix_state.view(-1, 4)[:, 0] < 0 if bt.prefix_mode else torch.zeros_like(on)
    live = on & ~done
    nc = bt.n_contrib.long()
    end_b = torch.minimum(nc, tc[:, 3][tile_of] + 1)
    zero = torch.zeros(T, dtype=torch.int64, device=tiles.device)
    fmax = zero.clone().scatter_reduce(0, tile_of[live], nc[live], "amax")
    bmax = zero.clone().scatter_reduce(0, tile_of[live], end_b[live], "amax")
    F = int(torch.clamp(fmax[tiles] - start_t[tiles], min=0).sum().item())
    Bn = int(torch.clamp(bmax[tiles] - start_t[tiles], min=0).sum().item())
    Pf = int((live & (nc > start_t[tile_of])).sum().item())
    Pb = int((live & (end_b > start_t[tile_of])).sum().item())
    S = big = 0
    if bt.layout == 1 and nt:
        off = bt.bin_offsets[: nt * 256].long().view(nt, 256)
        rng = bt.ranges.view(T, 2).long()
        bins = torch.cat([off, rng[tiles, 1:2]], 1)  # [nt, 257] bin starts, then the end
        walked = fmax[tiles] > start_t[tiles]
        first = rng[tiles, 0] + start_t[tiles]
        last = rng[tiles, 0] + torch.clamp(fmax[tiles], min=1) - 1
        b_lo = (torch.searchsorted(bins, first.view(-1, 1), right=True).view(-1) - 1).clamp(0, 255)
        b_hi = torch.maximum(
            (torch.searchsorted(bins, last.view(-1, 1), right=True).view(-1) - 1).clamp(0, 255),
            b_lo)
        lo = bins.gather(1, b_lo.view(-1, 1)).view(-1)
        hi = bins.gather(1, (b_hi + 1).view(-1, 1)).view(-1)
        S = int(torch.where(walked, hi - lo, torch.zeros_like(hi)).sum().item())
        size = bins[:, 1:] - bins[:, :-1]
        k = torch.arange(256, device=size.device).view(1, 256)
        inwin = (k >= b_lo.view(-1, 1)) & (k <= b_hi.view(-1, 1)) & walked.view(-1, 1)
        big = int(torch.where(inwin & (size > abi_lazy_max()), size,
                              torch.zeros_like(size)).sum().item())
    return {"rendered_tiles": nt, "rendered_pixels": int(on.sum().item()),
            "forward_entries": F, "backward_entries": Bn,
            "forward_pixels": Pf, "backward_pixels": Pb, "keys_sorted_by_forward": S,
            "keys_in_large_bins": big}


def _a256(x: int) -> int:
    return (x + 255) // 256 * 256


def proj_workspace_offsets(info) -> dict:
    """Byte offsets of the projection workspace's regions (the layout the
    binning entry point uses; their total is checked against
    cls_project_workspace_size by the host tests)."""
    V, T = int(info.n_views), int(info.total_tiles)
    cpv = (int(info.max_n) + 2047) // 2048
    sizes = [("partials", (cpv * V + 1) * 8), ("sat", info.total_sat * 4),
             ("diff", info.total_sat * 4), ("zmin", V * 4), ("zmax", V * 4),
             ("tile_rank", T * 4), ("cursor", T * 256 * 4),
             ("tile_partials", ((T + 63) // 64 + 1) * 8),
             ("big_list", info.total_records * 16), ("big_count", 4),
             ("sbins", 256 * info.total_sat * 4), ("abins", 256 * info.total_sat * 4),
             ("arange", V * 8), ("ttot", T * 4), ("work_list", info.total_records * 16),
             ("work_count", V * 8), ("front", T), ("t_win", T * 15 * 2), ("rank0", V * 4),
             ("compact", ((T + 4095) // 4096 + 1) * 8), ("rects", info.total_records * 16)]
    off, o = {}, 0
    for name, size in sizes:
        off[name] = o
        o = _a256(o + int(size))
    off["total"] = o
    return off


def occupied_grid_entries(bt) -> int:
    """Entries of the active Gaussians' depth-bin grid that one binning call
    prefix-sums and clears: per view its (Tx + 1)(Ty + 1) cells times the
    depth bins its active Gaussians occupy (read from the workspace)."""
    import torch
    off = proj_workspace_offsets(bt.info)
    V = bt.n_views
    ar = bt.proj_ws[off["arange"]: off["arange"] + 8 * V].view(torch.int32).cpu().numpy()
    lo, hi = ar[:V].view(np.uint32).astype(np.int64), ar[V:].view(np.uint32).astype(np.int64)
    total = 0
    for j in range(V):
        v = bt.view_tab[j]
        if hi[j] >= lo[j]:
            total += (int(v.tiles_x) + 1) * (int(v.tiles_y) + 1) * int(hi[j] - lo[j] + 1)
    return total


def design_bytes(lu):
    """Algorithmic DRAM bytes one iteration of this design moves, per stage,
    from one more pass's own counters (run after the timed region):

      A active Gaussians, V views, N records per view (every Gaussian), R
      parameter-row bytes (3 + 3 + 4 + 1 + 3 (l+1)^2 floats), Np pair-producing
      records, E pairs emitted (counted from the key buffer, pre-filled with a
      value no key takes), S keys in the depth bins the forward pass sorts (the
      bins from the one holding a tile's walk start to the one holding its last
      composited entry), F / B list entries the forward / backward pass needs
      per tile (walk start to the deepest pixel's last contributor; for the
      backward, to the tile's last active entry), Pr rendered pixels, Pb those
      the backward walks, Tr rendered tiles, G the summed-area grid entries
      (per view (Tx+1)(Ty+1)), Go the active depth-bin grid entries one call
      passes over (occupied_grid_entries). The static Gaussians' counts per
      (tile, bin) are built once per update (by the call that projects every
      Gaussian) and are not counted here.

      project_and_bin  A V (R + 48 + 16)       rows read, records and packed
                                               rectangles written
                       + N V 16 + Np 16        rectangles read by the count,
                                               work items (rectangle + record)
                                               written
                       + A V 32                active rectangles read, their
                                               four depth-bin stamps
                       + Go 16                 active depth-bin grid: row pass
                                               (read, write), column pass (read,
                                               clear) over the Go entries of the
                                               bins the active Gaussians occupy
                       + 5 x 256 Tr 4          per (tile, bin): static counts
                                               read, counts written and read,
                                               offsets and cursors written
                       + Np 16 + 8 E           emission: work items read, keys
                                               written
      sort (large bins)  16 per key in a bin above the forward's sort limit
      render_forward   16 S + 48 F             keys sorted in shared memory and
                                               written back, records staged
                       + 64 Pr                 target, image, T, last
                                               contributor, dL/dC, prefix state
      render_backward  56 B + 44 Pb            keys and records, pixel state
                       + 16 (Pr - Pb)          prefix state of pixels not walked
                       + A V 48 3 + 2 A R      2D gradients (clear, sum, read),
                                               parameter rows and gradients
      adam             A 7 R                   theta, m, v read and written, g read
    """
    import torch
    bt = lu.batch
    st = lu.state
    V = bt.n_views
    A = st.n_active
    row = 4 * (11 + 3 * (st.sh_degree + 1) ** 2)
    bt.keys.fill_(-1)
    lu.render_pass(with_backward=True, with_adam=True)
    torch.cuda.synchronize()
    bt.check_status()
    n = min(int(bt.n_pairs.item()), bt.capacity)
    E = int((bt.keys[:n] != -1).sum().item())
    w = walk_counts(bt)
    nt, F, Bn, Pf, Pb, S, big = (w[k] for k in ("rendered_tiles", "forward_entries",
                                                "backward_entries", "forward_pixels",
                                                "backward_pixels", "keys_sorted_by_forward",
                                                "keys_in_large_bins"))
    Pr = w["rendered_pixels"]
    Np = pair_producing_records(bt)
    N = sum(bt.scenes[bt.view_tab[j].scene].n for j in range(V))
    G = int(bt.info.total_sat)
    Go = occupied_grid_entries(bt)
    stages = {
        "project_and_bin": A * V * (row + 64) + N * 16 + Np * 16 + A * V * 32 + Go * 16 +
        5 * 256 * nt * 4 + Np * 16 + 8 * E,
        "sort_keys": 16 * big,
        "render_forward": 16 * S + 48 * F + 64 * Pr,
        "render_backward": 56 * Bn + 44 * Pb + 16 * (Pr - Pb) + A * V * 48 * 3 + 2 * A * row,
        "adam_step_active": 7 * A * row,
    }
    counters = {"active": A, "views": V, "records": N, "pair_producing_records": Np,
                "pairs_emitted": E, "pairs_counted": int(bt.n_pairs.item()),
                "keys_sorted_by_forward": S, "keys_in_large_bins": big,
                "forward_entries": F, "backward_entries": Bn, "forward_pixels": Pf,
                "backward_pixels": Pb, "rendered_pixels": Pr, "rendered_tiles": nt,
                "sat_entries": G, "active_bin_grid_entries": Go,
                "row_bytes": row}
    return stages, counters


def abi_lazy_max():
    from paper_2506_21117_gb300 import _abi
    return _abi.LAZY_MAX_BIN


def executed_evaluations(bt):
    """(pixel, list entry) evaluations the render kernels execute in one pass:
    per pixel, the entries of its walk that the tile cull keeps (entries no
    pixel of the tile can reach with alpha >= 1/255 are dropped while a batch
    is staged and never evaluated). The cull is re-evaluated here in float32
    with the kernels' formula; `walked_evaluations` counts the same walks with
    the culled entries included. Bucketed layout only (None otherwise)."""
    import torch
    if bt.layout != 1:
        return None
    dev = bt.n_contrib.device
    T = bt.info.total_tiles
    nt = int(bt.n_active_tiles.item())
    tiles = bt.active_tiles[:nt].long()
    tile_of = _tile_maps(bt)
    tc = bt.tile_cache.view(T, 4).long()
    start_t = torch.where(tc[:, 1] == -1, torch.zeros_like(tc[:, 1]), tc[:, 1])
    rendered = torch.zeros(T, dtype=torch.bool, device=dev)
    rendered[tiles] = True
    done = bt.prefix_state.view(-1, 4)[:, 0] < 0 if bt.prefix_mode else torch.zeros_like(rendered[tile_of])
    live = rendered[tile_of] & ~done
    nc = bt.n_contrib.long()
    end_b = torch.minimum(nc, tc[:, 3][tile_of] + 1)
    fmax = torch.zeros(T, dtype=torch.int64, device=dev).scatter_reduce(
        0, tile_of[live], nc[live], "amax")
    lens = torch.clamp(fmax - start_t, min=0)
    lens = torch.where(rendered, lens, torch.zeros_like(lens))
    offs = torch.cumsum(lens, 0) - lens
    total = int(lens.sum().item())
    if total == 0:
        return {"forward": 0, "backward": 0, "kept_share": 0.0}
    tid = torch.repeat_interleave(torch.arange(T, device=dev), lens)
    pos = torch.arange(total, device=dev) - offs[tid] + start_t[tid]
    rng = bt.ranges.view(T, 2).long()
    key = bt.keys[rng[tid, 0] + pos]
    rec = (key & 0xFFFFFFFF).long()
    r = bt.records.view(-1, 12)[rec]
    u, v, A, B, C, o = (r[:, i] for i in range(6))
    tx0 = torch.zeros(T, dtype=torch.float32, device=dev)
    ty0 = torch.zeros(T, dtype=torch.float32, device=dev)
    for j in range(bt.n_views):
        vw = bt.view_tab[j]
        n = int(vw.tiles_x) * int(vw.tiles_y)
        loc = torch.arange(n, device=dev)
        tx0[int(vw.tile_base): int(vw.tile_base) + n] = (loc % int(vw.tiles_x)).float() * 16
        ty0[int(vw.tile_base): int(vw.tile_base) + n] = (loc // int(vw.tiles_x)).float() * 16
    X0 = (tx0[tid] + 0.5) - u
    X1 = (tx0[tid] + 15.5) - u
    Y0 = (ty0[tid] + 0.5) - v
    Y1 = (ty0[tid] + 15.5) - v
    inside = (X0 <= 0) & (X1 >= 0) & (Y0 <= 0) & (Y1 >= 0)

    def clamp(x, lo, hi):
        return torch.minimum(torch.maximum(x, lo), hi)
    ya = clamp(-B * X0 / C, Y0, Y1)
    yb = clamp(-B * X1 / C, Y0, Y1)
    xa = clamp(-B * Y0 / A, X0, X1)
    xb = clamp(-B * Y1 / A, X0, X1)
    q = torch.minimum(torch.minimum(A * X0 * X0 + 2 * B * X0 * ya + C * ya * ya,
                                    A * X1 * X1 + 2 * B * X1 * yb + C * yb * yb),
                      torch.minimum(A * xa * xa + 2 * B * xa * Y0 + C * Y0 * Y0,
                                    A * xb * xb + 2 * B * xb * Y1 + C * Y1 * Y1))
    DX = torch.maximum(X0.abs(), X1.abs())
    DY = torch.maximum(Y0.abs(), Y1.abs())
    S = (A.abs() + B.abs()) * DX * DX + (B.abs() + C.abs()) * DY * DY
    q_lo = q - 1e-5 * S - 1e-5
    culled = (o < (1.0 / 255.0) * 0.999) | (~inside & (q_lo > 2.0 * torch.log(o * (255.0 / 0.999))))
    cum = torch.cat([torch.zeros(1, dtype=torch.int64, device=dev),
                     torch.cumsum((~culled).long(), 0)])

    def count(ends):
        t = tile_of
        ok = live & (ends > start_t[t])
        e = torch.clamp(ends, max=fmax[t])
        a = offs[t]
        b = offs[t] + (e - start_t[t])
        return int(torch.where(ok, cum[b.clamp(min=0)] - cum[a], torch.zeros_like(a)).sum().item())
    return {"forward": count(nc), "backward": count(end_b),
            "kept_share": float((~culled).float().mean().item())}


PROFILE_OF_STAGE = {"render_backward": ("render_bwd_1M_4x1080p.md", "csrc/render_bwd.cu"),
                    "render_forward": ("render_fwd_1M_4x1080p.md", "csrc/render_fwd.cu")}


def profiled_traffic(stage: str, args):
    """DRAM bytes per launch of a stage's kernel from the committed ncu summary,
    only if the summary was taken on this workload and on the current kernel
    source (else None)."""
    import hashlib
    default = (args.n, args.width, args.height, args.views, args.fraction) == \
        (1_000_000, 1920, 1080, 4, 0.05)
    if stage not in PROFILE_OF_STAGE or not default:
        return None
    md, src = PROFILE_OF_STAGE[stage]
    try:
        text = open(os.path.join(ROOT, "profiles", md)).read()
        m = hashlib.sha256()
        for f in (src, "csrc/common.cuh"):
            m.update(open(os.path.join(ROOT, "paper_2506_21117_gb300", f), "rb").read())
        if f"source_sha256_16: {m.hexdigest()[:16]}" not in text:
            return None
        for line in text.splitlines():
            if line.startswith("dram_bytes_per_launch:"):
                return int(line.split(":")[1])
    except OSError:
        return None
    return None


def max_over_ranks(x: float, device=None) -> float:
    """The largest value of `x` over all ranks (the whole job's time)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, steps: int, max_ms: float) -> float:
    """Iterations of all ranks per second of the slowest rank (weak scaling:
    every rank runs its own update)."""
    return world * steps / (max_ms / 1e3)


def setup_workload(args, seed):
    from paper_2506_21117_gb300 import synthetic as S
    return S.workload_large(n=args.n, n_views=args.views, width=args.width, height=args.height,
                            fraction=args.fraction, sh_degree=3, seed=seed)


# -------------------------------------------------------------- CPU oracle ---

ORACLE_TILES = 64        # active tiles per oracle sample, drawn over every view
ORACLE_PROJ_FRAC = 0.05  # share of the Gaussians projected (with backward) per sample


def oracle_sample(scene, cams, targets, active, seed=0, cache=None):
    """Time the float64 oracle, single-threaded, on a bounded sample of one
    iteration of the workload: the float32 index projection plus the float64
    projection with its backward for ORACLE_PROJ_FRAC of the Gaussians in
    every view, and forward + backward (lists cut where every pixel stopped)
    of ORACLE_TILES active tiles drawn at random over all views, each over
    the Gaussians whose rectangles reach it. Extrapolated to every Gaussian
    and every active tile. Returns (seconds per iteration, description). The
    benchmark's cpu_baseline and the reference arm use this same sample."""
    import torch
    from oracle import fp32_index as fx
    from oracle import projection as pj
    from oracle import step as ostep
    cache = {} if cache is None else cache
    n = scene["means"].shape[0]
    rng = np.random.default_rng(seed)
    if "tiles" not in cache:  # set-up, not timed
        cache["pidx"] = [fx.project_index(scene, c) for c in cams]
        cache["tiles"] = []
        for j, (p, c) in enumerate(zip(cache["pidx"], cams)):
            ys, xs = np.nonzero(fx.tile_mask(p, active, c))
            cache["tiles"] += [(j, int(x), int(y)) for x, y in zip(xs, ys)]
    all_tiles = cache["tiles"]
    pick = [all_tiles[i] for i in rng.choice(len(all_tiles), size=min(ORACLE_TILES,
                                                                         len(all_tiles)),
                                                replace=False)]
    m = max(1, int(n * ORACLE_PROJ_FRAC))
    start = int(rng.integers(0, n - m + 1))
    sub = {k: v[start:start + m] for k, v in scene.items()}
    threads = torch.get_num_threads()
    torch.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        for c in cams:
            fx.project_index(sub, c)
            g = pj.scene64(sub, requires_grad=True)
            P = pj.project(g, c, 3)
            (P["u"].sum() + P["conic"].sum() + P["rgb"].sum()).backward()
        t_proj = (time.perf_counter() - t0) * (n / m)
        t_tiles = 0.0
        for j in range(len(cams)):
            mine = [(x, y) for (v, x, y) in pick if v == j]
            if not mine:
                continue
            p = cache["pidx"][j]
            sel = np.zeros(n, bool)
            for (tx, ty) in mine:
                sel |= p["valid"] & (p["tx0"] <= tx) & (p["tx1"] >= tx) & (p["ty0"] <= ty) & \
                    (p["ty1"] >= ty)
            subs = {k: v[sel] for k, v in scene.items()}
            t1 = time.perf_counter()
            ostep.render(subs, cams[j:j + 1], 3, targets=targets[j:j + 1], loss="l1",
                         need_grad=True, tiles=[mine], truncate=True)
            t_tiles += time.perf_counter() - t1
    finally:
        torch.set_num_threads(threads)
    per_tile = t_tiles / max(len(pick), 1)
    it = t_proj + len(all_tiles) * per_tile
    desc = (f"float64 oracle on 1 thread, one iteration extrapolated from: index + float64 "
            f"projection with backward of {m} of {n} Gaussians in each of {len(cams)} views "
            f"(x{n / m:.0f}) and forward + backward of {len(pick)} active tiles drawn over all "
            f"views, over the Gaussians reaching them (x{len(all_tiles) / max(len(pick), 1):.0f} "
            f"to all {len(all_tiles)} active tiles)")
    return it, desc


def cpu_fp32_iterations(scene, cams, targets, active, iters=2, loss="l1", sh_degree=3):
    """The float32 OpenMP CPU baseline (the plain algorithm: every list built
    and sorted each iteration, active tiles only) on all host cores: `iters`
    full iterations (forward, backward, masked Adam), timed whole."""
    from oracle import cpu_baseline as cb
    cores = os.cpu_count() or 1
    b = cb.Baseline(scene, cams, sh_degree, targets, active, loss, threads=cores)
    t0 = time.perf_counter()
    for _ in range(iters):
        b.iteration()
    dt = time.perf_counter() - t0
    return iters / dt, cores


# ---------------------------------------------------------------- our arm ---

def run_ours(args, rank, world):
    import torch
    from paper_2506_21117_gb300 import build as b
    b.build()
    from paper_2506_21117_gb300.update import LocalUpdate
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)

    scene, target_scene, cams, masks, box = setup_workload(args, seed=rank)
    n = scene["means"].shape[0]
    # target images: full renders of the changed scene with this library
    tgt = LocalUpdate(target_scene, cams, 3, active=np.ones(n, bool), capacity_slack=1.05)
    tgt.render_pass(with_backward=False)
    torch.cuda.synchronize()
    tgt.batch.check_status()
    targets = [t.cpu().numpy().copy() for t in tgt.batch.per_view(tgt.batch.image, 3)]
    del tgt
    torch.cuda.empty_cache()

    lu = LocalUpdate(scene, cams, 3, targets=targets, masks=masks, loss=args.loss)
    ssim = args.loss == "l1+ssim"
    bt = lu.batch
    A = lu.state.n_active
    clocks = Clocks(dev.index)
    for _ in range(args.warmup):
        lu.step()
    torch.cuda.synchronize()
    bt.check_status()
    if args.profile_iteration:
        torch.cuda.nvtx.range_push("cls_iteration")
        lu.render_pass(with_backward=True, with_adam=True)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        bt.check_status()
        clocks.stop(0.0, 0.0)
        return {"profile_iteration": True, "workload": WORKLOAD, "n_gaussians": n,
                "active_gaussians": A, "launches": bt.launches_per_step()}

    stages = ["project_and_bin", "sort_keys", "render_forward"] + (["ssim_loss"] if ssim else []) + \
        ["render_backward", "adam_step_active"]
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(stages) + 1)]
          for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record()
    for k in range(args.steps):
        e = ev[k]
        e[0].record()
        bt.project_and_bin(1)
        e[1].record()
        bt.sort()
        e[2].record()
        bt.render(lu.loss_mode, lu.bg)
        i = 3
        e[i].record()
        if ssim:
            bt.apply_ssim(lu.loss_mode)
            i += 1
            e[i].record()
        bt.backward()
        e[i + 1].record()
        bt.adam(lu.lr)
        e[i + 2].record()
    end.record()
    torch.cuda.synchronize()
    eager_ms = start.elapsed_time(end)
    # the same iterations replayed from a CUDA graph (the value reported)
    graph = lu.capture()
    for _ in range(args.warmup):
        graph.replay()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_val0 = time.time()
    start.record()
    for k in range(args.steps):
        graph.replay()
    end.record()
    torch.cuda.synchronize()
    t_val1 = time.time()
    total_ms = max_over_ranks(start.elapsed_time(end), dev)
    # the same replay held for about two seconds, so that many clock samples
    # fall inside one window (the K-step window above is tens of ms)
    n_sus = max(args.steps, int(math.ceil(2000.0 / max(total_ms / args.steps, 1e-3))))
    t_sus0 = time.time()
    start.record()
    for k in range(n_sus):
        graph.replay()
    end.record()
    torch.cuda.synchronize()
    t_sus1 = time.time()
    sus_ms = start.elapsed_time(end)
    clk_all = clocks.stop(t_wall0, t_sus1)
    clk = clocks.window(t_val0, t_val1)
    clk_sus = clocks.window(t_sus0, t_sus1)
    bt.check_status()
    stage_ms = {s: sum(ev[k][i].elapsed_time(ev[k][i + 1]) for k in range(args.steps)) / args.steps
                for i, s in enumerate(stages)}

    # counters of one more pass (not timed)
    bt.n_contrib.zero_()
    lu.render_pass(with_backward=False)
    torch.cuda.synchronize()
    D = int(bt.n_pairs.item())
    tiles_on = int(bt.n_active_tiles.item())
    walked = walked_evaluations(bt)
    V = len(cams)
    passes = math.ceil(bt.info.key_bits / 8)
    P_act = tiles_on * 256
    ssim_roof = None
    if ssim:
        # pass 1 reads x, y (24 B) and writes a, b, c (36 B) per rendered pixel;
        # pass 2 reads a, b, c, x, y and dL/dC and writes dL/dC (84 B) per covered pixel
        covered = int((bt.tile_active == 1).sum().item()) * 256
        b_ssim = 60 * P_act + 84 * covered
        ach = b_ssim / (stage_ms["ssim_loss"] * 1e-3) / 1e9
        ssim_roof = {"bound": "hbm", "bytes_per_launch": b_ssim, "achieved": ach,
                     "unit": "GB/s", "rendered_pixels": P_act, "covered_pixels": covered}
    stage_bytes, counters = design_bytes(lu)
    if ssim:
        stage_bytes["ssim_loss"] = ssim_roof["bytes_per_launch"]

    ms_per_step = total_ms / args.steps
    value = whole_job_rate(world, args.steps, total_ms)
    hbm_peak, peak_kind, sm_max = load_peaks()
    # the dominant single kernel is a render kernel (project_and_bin is a stage
    # of some twenty short kernels, the largest under half a render kernel)
    dominant = max(("render_forward", "render_backward"), key=stage_ms.get)
    alu_peak = fp32_peak_tflops(sm_max)
    executed = executed_evaluations(bt)
    counted = executed if executed is not None else walked
    evals = counted["forward" if dominant == "render_forward" else "backward"]
    flops = evals * (FWD_FLOP_PER_EVAL if dominant == "render_forward" else BWD_FLOP_PER_EVAL)
    ach = flops / (stage_ms[dominant] * 1e-3) / 1e12
    roof = {"kernel": dominant, "bound": "alu", "achieved": ach, "peak": alu_peak,
            "unit": "TFLOP/s", "frac": ach / alu_peak,
            "traffic": profiled_traffic(dominant, args),
            "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock",
            "units_per_launch": evals,
            "unit_work": "(pixel, list entry) evaluations executed: walked after the cached "
                         "prefix, entries the tile cull drops excluded",
            "evaluations_executed": executed, "evaluations_walked": walked,
            "hbm_of_stage": {"bytes": stage_bytes[dominant],
                             "achieved_gbs": stage_bytes[dominant] / (stage_ms[dominant] * 1e-3)
                             / 1e9}}
    roof["hbm_of_stage"]["frac"] = roof["hbm_of_stage"]["achieved_gbs"] / hbm_peak
    # the whole iteration against HBM: this design's own bytes (design_bytes)
    # per replayed iteration; per stage against its eager event time
    B_iter = sum(stage_bytes.values())
    per_iter_s = ms_per_step * 1e-3
    iteration_roof = {
        "bytes_per_iter": B_iter, "achieved_gbs": B_iter / per_iter_s / 1e9,
        "peak_gbs": hbm_peak, "peak_kind": peak_kind,
        "frac": B_iter / per_iter_s / 1e9 / hbm_peak,
        "basis": "algorithmic bytes of this design (bucketed binning, lazy per-bin sort, "
                 "cached static prefix), from the pass's own counters",
        "stages": {k: {"bytes": b, "ms": stage_ms.get(k),
                       "gbs": (b / (stage_ms[k] * 1e-3) / 1e9) if stage_ms.get(k) else None}
                   for k, b in stage_bytes.items()},
        "counters": counters,
    }
    # the survey's formula for a design with a global radix sort of every
    # counted pair (12 B x pairs x (2 passes + 1)): bytes this design avoids
    B_global = (A * (236 + 48 * V) + 12 * D * (2 * passes + 1) + 2 * 48 * D +
                P_act * (12 + 8 + 12 + 12 + 8) + A * (36 * V + 236 + 236) + 28 * 59 * A)
    iteration_roof["global_sort_equivalent"] = {
        "bytes_per_iter": B_global, "achieved_gbs": B_global / per_iter_s / 1e9,
        "frac": B_global / per_iter_s / 1e9 / hbm_peak,
        "note": "bytes a global-sort design would move for the same pairs; not moved here"}

    e2e = run_e2e(args, lu, targets, masks, cams)
    active_np = lu.state.active.cpu().numpy().astype(bool)
    sphere = run_sphere_region(lu)
    densify = run_densify(lu)
    sampling = run_sampling()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step,
        "execution": "CUDA graph replay of one captured iteration",
        "eager_ms_per_step": eager_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_gaussians": n, "views": V,
                   "resolution": f"{args.width}x{args.height}", "sh_degree": 3,
                   "change_fraction": args.fraction, "active_gaussians": A,
                   "active_tiles": tiles_on, "pairs": D, "sort_passes": passes,
                   "parallelism": f"replicas x{world} (independent scenes, no collective)",
                   "l2": "inputs larger than L2 (params 256 MB, keys >= 100 MB per step)"},
        "stages_ms": stage_ms,
        "roofline": roof,
        "iteration_hbm_roofline": iteration_roof,
        "clocks": clk,
        "sustained": {"iterations": n_sus, "ms_per_step": sus_ms / n_sus,
                      "value": n_sus / (sus_ms * 1e-3) * world, "clocks": clk_sus,
                      "ms_x_sm_mhz": (sus_ms / n_sus) * (clk_sus["sm_mhz"] or float("nan")),
                      "note": "the same graph replay held ~2 s after the timed K steps"},
        "clocks_whole_run": clk_all,
        "e2e": e2e,
        "gpu_launches": int(bt.launches_per_step() * args.steps),
        "sphere_region": sphere,
        "densification": densify,
        "new_point_sampling": sampling,
    }
    if ssim_roof is not None:
        ssim_roof["peak"] = hbm_peak
        ssim_roof["frac"] = ssim_roof["achieved"] / hbm_peak
        line["ssim_roofline"] = ssim_roof
        line["config"]["workload"] = WORKLOAD.replace(", L1", ", L1 + D-SSIM (0.8/0.2)")
    if not args.no_serving:
        del lu, bt
        torch.cuda.empty_cache()
        line["serving"] = run_serving(args, seed=rank)
    if not args.no_configs:
        line["other_configs"] = run_configs(args)
        line["active_fraction_sweep"] = run_sweep(args, rank)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sec, desc = oracle_sample(scene, cams, targets, active_np, seed=0)
        line["cpu_baseline"] = {"value": 1.0 / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": desc}
        rate, cores = cpu_fp32_iterations(scene, cams, targets, active_np, iters=2)
        line["cpu_fp32_baseline"] = {
            "value": rate, "unit": UNIT, "cores": cores,
            "kind": "float32 OpenMP plain algorithm (oracle/cpu_fp32.cpp)",
            "sample": "2 full iterations of the benchmark workload (forward, backward, masked "
                      "Adam; every active tile's list built and sorted each iteration)"}
    return line


def _replay_rate(lu, steps: int, warmup: int = 5):
    """Iterations per second of a captured iteration replayed `steps` times
    (after `warmup` eager iterations), CUDA events around the replays."""
    import torch
    for _ in range(warmup):
        lu.step()
    g = lu.capture()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        g.replay()
    b.record()
    torch.cuda.synchronize()
    lu.batch.check_status()
    ms = a.elapsed_time(b) / steps
    return {"iters_per_s": 1e3 / ms, "ms_per_iter": ms, "replays": steps}


def _target_images(scene, cams, sh_degree):
    """Full renders of a scene with this library (the update's targets)."""
    import torch
    from paper_2506_21117_gb300.update import LocalUpdate
    n = scene["means"].shape[0]
    t = LocalUpdate(scene, cams, sh_degree, active=np.ones(n, bool), capacity_slack=1.05)
    t.render_pass(with_backward=False)
    torch.cuda.synchronize()
    t.batch.check_status()
    out = [x.cpu().numpy().copy() for x in t.batch.per_view(t.batch.image, 3)]
    del t
    torch.cuda.empty_cache()
    return out


def run_configs(args):
    """GPU timings of the other workloads, each in the launch configuration
    of the benchmark (bucketed binning, lazy sort, cached prefix, CUDA-graph
    replay): the plain render + backward + Adam (2,000 Gaussians, one 64x64
    view, L1, all active), the local update (100,000 Gaussians, SH 3, eight
    800x800 views, 5% box: lifting, planning and 30 iterations, wall clock,
    plus the replay rate), the finite-difference workload (500 Gaussians,
    SH 1, two 32x32 views, L2, all active)."""
    import torch
    from paper_2506_21117_gb300 import synthetic as S
    from paper_2506_21117_gb300.update import LocalUpdate
    out = {}
    scene, cams, targets = S.workload_plain()
    lu = LocalUpdate(scene, cams, 0, targets=targets, active=np.ones(2000, bool), loss="l1")
    out["plain_2k_64x64_l1"] = _replay_rate(lu, 500)
    scene, cams, targets = S.workload_fd()
    lu = LocalUpdate(scene, cams, 1, targets=targets, active=np.ones(500, bool), loss="l2")
    out["fd_500_2x32x32_l2"] = _replay_rate(lu, 500)
    scene, target_scene, cams, masks, _ = S.workload_local(n=100_000, n_views=8, size=800)
    targets = _target_images(target_scene, cams, 3)
    LocalUpdate(scene, cams, 3, targets=targets, masks=masks, loss="l1").run(3)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lu = LocalUpdate(scene, cams, 3, targets=targets, masks=masks, loss="l1")
    lu.run(30)
    loss = float(lu.batch.loss[0].item())
    wall = time.perf_counter() - t0
    rate = _replay_rate(lu, 200, warmup=0)
    out["local_100k_8x800_30it"] = {
        "update_wall_ms": wall * 1e3, "iters_per_s_incl_lift_and_plan": 30 / wall,
        "replay": rate, "active_gaussians": lu.state.n_active,
        "active_tiles": int(lu.batch.n_active_tiles.item()), "loss_after_30": loss}
    del lu
    torch.cuda.empty_cache()
    return out


def run_sweep(args, rank):
    """The benchmark workload with change boxes holding 1% and 10% of the
    Gaussians (5% is the headline): replay rate and eager stage times."""
    import torch
    from paper_2506_21117_gb300.update import LocalUpdate
    out = {}
    for frac in (0.01, 0.10):
        a = argparse.Namespace(**vars(args))
        a.fraction = frac
        scene, target_scene, cams, masks, _ = setup_workload(a, seed=rank)
        targets = _target_images(target_scene, cams, 3)
        lu = LocalUpdate(scene, cams, 3, targets=targets, masks=masks, loss="l1")
        rate = _replay_rate(lu, 100, warmup=10)
        bt = lu.batch
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        tot = [0.0] * 5
        for _ in range(20):
            ev[0].record()
            bt.project_and_bin(1)
            ev[1].record()
            bt.sort()
            ev[2].record()
            bt.render(lu.loss_mode, lu.bg)
            ev[3].record()
            bt.backward()
            ev[4].record()
            bt.adam(lu.lr)
            ev[5].record()
            torch.cuda.synchronize()
            for i in range(5):
                tot[i] += ev[i].elapsed_time(ev[i + 1]) / 20
        out[f"{int(round(frac * 100))}%"] = {
            **rate, "active_gaussians": lu.state.n_active,
            "active_tiles": int(bt.n_active_tiles.item()),
            "stages_ms_eager": dict(zip(["project_and_bin", "sort_keys", "render_forward",
                                          "render_backward", "adam_step_active"], tot))}
        del lu, bt
        torch.cuda.empty_cache()
    return out


def run_sphere_region(lu):
    """Sphere region of the benchmark's O^t (K-Means, spheres) and one pruning
    check, timed with CUDA events on the launching stream (after the timed
    iterations; the pruning check removes the Gaussians that left it)."""
    import torch
    from paper_2506_21117_gb300.update import SphereRegion, prune_outside
    st = lu.state
    A = st.n_active
    SphereRegion(st)  # warm-up (first launch of each kernel)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record()
    region = SphereRegion(st)
    e[1].record()
    e[2].record()
    removed = prune_outside(st, region)
    e[3].record()
    torch.cuda.synchronize()
    return {"active_gaussians": A, "spheres": region.k, "kmeans_iters": 16,
            "fit_ms": e[0].elapsed_time(e[1]), "prune_check_ms": e[2].elapsed_time(e[3]),
            "removed": removed, "note": "prune_check_ms includes reading the removed count back"}


def run_densify(lu):
    """Densification of the benchmark's O^t (base 3DGS adaptive density
    control restricted to O^t): the per-iteration statistics pass, one
    densification step (clone/split/prune, reading its counts back) and the
    rebuild of the batch for the grown scene; CUDA events on the launching
    stream, the rebuild by wall clock."""
    import torch
    from paper_2506_21117_gb300 import synthetic as S
    from paper_2506_21117_gb300.densify import Densifier
    st = lu.state
    A0 = st.n_active
    d = Densifier(st, lu.cams, S.densify_draws(0))
    lu.batch.refresh_active()  # the pruning check above may have shrunk O^t
    lu.render_pass(True, False)
    d.accumulate(lu.batch)  # warm-up
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record()
    d.accumulate(lu.batch)
    e[1].record()
    torch.cuda.synchronize()
    e[2].record()
    added, removed = d.densify(3000)
    e[3].record()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lu._rebuild_batch()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    return {"active_gaussians": A0, "accumulate_ms": e[0].elapsed_time(e[1]),
            "densify_ms": e[2].elapsed_time(e[3]), "rebuild_ms": (t1 - t0) * 1e3,
            "added": added, "removed": removed, "active_after": st.n_active,
            "note": "statistics of two iterations; densify_ms includes reading the counts back"}


def run_sampling():
    """New-point sampling for an appearing object at the local-update size
    (100k Gaussians, 8 views of 800x800, the Gaussians of a 5% box removed),
    from an empty O to 5000 points (box round, then K-Means mixture rounds, each
    filtered by the vote), then the new Gaussians' initialisation; wall time
    of the host-driven rounds (each reads the kept count back)."""
    import torch
    from paper_2506_21117_gb300 import synthetic as S
    from paper_2506_21117_gb300.sampling import init_gaussians, sample_points
    from paper_2506_21117_gb300.update import SceneState
    scene, cams, masks, _ = S.workload_addition(n=100_000, n_views=8, size=800, seed=0)
    st = SceneState(scene, 3)
    st.set_active(np.zeros(st.n, bool))
    masks_dev = torch.from_numpy(np.concatenate([m.reshape(-1) for m in masks])).cuda()
    draws = S.sampling_draws(0)
    sample_points(st, cams, masks_dev, 500, draws)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = sample_points(st, cams, masks_dev, 5000, draws)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    rows = init_gaussians(out["new"], 3)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    return {"workload": "100k Gaussians, 8 views 800x800, empty 5% box, target 5000 points",
            "points": int(out["points"].shape[0]), "rounds": out["rounds"],
            "sample_ms": (t1 - t0) * 1e3, "init_ms": (t2 - t1) * 1e3,
            "new_gaussians": int(rows.shape[0])}


def run_serving(args, seed=0):
    """Serving workload: resident scenes with log-uniform sizes, Poisson update
    requests (2-8 views at 640x480, 800x800 or 1280x720, a change box holding
    1-10% of the scene, 10 local iterations each), continuous batching against
    the plain one-at-a-time loop on the same kernels (the batched loop holds
    new admissions while its composition is younger than three steps, unless
    enough requests wait to fill every free slot). Saturation first (all
    requests queued at once); then open-loop Poisson streams at the configured
    rate (30 s by default, if below the batched saturation rate) and at 50% and
    90% of the batched saturation rate (10 s each)."""
    import torch
    from paper_2506_21117_gb300 import synthetic as S
    from paper_2506_21117_gb300.serving import Request, Server, run_plain
    from paper_2506_21117_gb300.update import SceneState
    t_setup = time.perf_counter()
    scenes, centres = S.serving_scenes(args.serving_scenes, seed=seed)
    templates = S.serving_templates(scenes, centres, 32, seed=seed)
    states = [SceneState(sc, 3) for sc in scenes]
    del scenes
    rng = np.random.default_rng(seed + 40)
    tgt = {}
    for (W, H) in S.SERVING_RESOLUTIONS:
        img = rng.uniform(0, 1, size=(8, 3, H, W)).astype(np.float32)
        tgt[(W, H)] = torch.from_numpy(img.reshape(-1)).pin_memory()
    packed = []
    for tp in templates:
        W, H = int(tp["cams"][0]["width"]), int(tp["cams"][0]["height"])
        V = len(tp["cams"])
        m = torch.from_numpy(np.concatenate([x.reshape(-1) for x in tp["masks"]])).pin_memory()
        packed.append((tp["scene"], tp["cams"], m, tgt[(W, H)][: V * 3 * H * W]))
    setup_s = time.perf_counter() - t_setup

    def requests(schedule):
        return [Request(rid=i, scene=packed[k][0], cams=packed[k][1], masks=packed[k][2],
                        targets=packed[k][3], iters=10, arrival=t) for i, (t, k) in enumerate(schedule)]

    n_sat = 96
    sat_sched = [(0.0, int(rng.integers(0, len(packed)))) for _ in range(n_sat)]
    warm = requests(sat_sched[:8])
    Server(states, max_slots=args.serving_slots, admit_interval=3).serve(warm, realtime=False)
    sat_b = Server(states, max_slots=args.serving_slots, admit_interval=3).serve(requests(sat_sched), realtime=False)
    sat_p = run_plain(states, requests(sat_sched[: n_sat // 2]), realtime=False)
    # the configured rate (if the batched loop can sustain it), then 50% and
    # 90% of the batched saturation rate (at 90% the plain loop is past its
    # own capacity)
    sat_rate = sat_b["updates_per_s"]
    points = []
    if args.serving_rate < sat_rate:
        points.append((args.serving_rate, args.serving_seconds, "configured"))
    points += [(0.5 * sat_rate, args.serving_load_seconds, "50% of batched saturation"),
               (0.9 * sat_rate, args.serving_load_seconds, "90% of batched saturation")]
    open_loop = []
    for rate, secs, what in points:
        sched = S.poisson_arrivals(rate, secs, len(packed), seed=seed + int(rate))
        cut = 2.0 * secs
        b = Server(states, max_slots=args.serving_slots, admit_interval=3).serve(requests(sched), realtime=True,
                                                              deadline=cut)
        p = run_plain(states, requests(sched), realtime=True, deadline=cut)
        open_loop.append({"rate_per_s": rate, "point": what, "seconds": secs,
                          "requests": len(sched), "deadline_s": cut, "batched": b, "plain": p})
    return {"scenes": len(states), "setup_s": setup_s, "templates": len(packed),
            "iters_per_update": 10, "slots": args.serving_slots,
            "saturation": {"batched": sat_b, "plain": sat_p},
            "open_loop": open_loop}


def run_e2e(args, lu, targets, masks, cams):
    """End to end through the public update API: every step is one scene update
    on the resident scene: pinned host targets and masks copied to the device,
    change-mask lifting, planning, `iters_per_update` iterations, the loss read
    back to the host. A first, untimed update builds its batch (tables and
    buffers for this scene and these views: a one-time cost per set of views,
    timed apart as `new_batch_update_ms`); the timed updates each take over the
    previous update's batch (`LocalUpdate.from_resident(reuse=...)`)."""
    import torch
    from paper_2506_21117_gb300.update import LocalUpdate
    tg = torch.from_numpy(np.concatenate([t.reshape(-1) for t in targets])).pin_memory()
    mk = torch.from_numpy(np.concatenate([m.reshape(-1) for m in masks])).pin_memory()
    state = lu.state
    h2d = tg.numel() * 4 + mk.numel()
    its = args.iters_per_update
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    u = LocalUpdate.from_resident(state, cams, tg, mk, loss="l1")  # builds its own batch
    u.run(its)
    loss = float(u.batch.loss[0].item())
    torch.cuda.synchronize()
    first_ms = (time.perf_counter() - t0) * 1e3
    t0 = time.perf_counter()
    for _ in range(args.e2e_updates):
        # each update takes over the previous one's batch (same scene, same views)
        u = LocalUpdate.from_resident(state, cams, tg, mk, loss="l1", reuse=u)
        u.run(its)
        loss = float(u.batch.loss[0].item())
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"value": args.e2e_updates * its / dt, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": 4, "step": f"one scene update of {its} iterations",
            "updates_timed": args.e2e_updates, "new_batch_update_ms": first_ms,
            "loss": loss}


def run_cpu_configs(args):
    """The float64 oracle on one thread and the float32 OpenMP baseline on all
    host cores, on the other workloads, in full: the plain render + backward
    (2,000 Gaussians, 64x64, L1), the finite-difference workload (500
    Gaussians, two 32x32 views, L2), and the 100k local update (8 views of
    800x800; the oracle one iteration over the tiles O^t touches, whose
    gradients equal the full image's; the baseline all 30 iterations)."""
    import torch
    from oracle import fp32_index as fx
    from oracle import step as ostep
    from paper_2506_21117_gb300 import synthetic as S
    out = {}
    torch.set_num_threads(1)

    def oracle_time(scene, cams, deg, targets, active, loss, tiles=None):
        t0 = time.perf_counter()
        ostep.render(scene, cams, deg, targets=targets, loss=loss, need_grad=True, tiles=tiles,
                     truncate=True)
        return time.perf_counter() - t0

    scene, cams, targets = S.workload_plain()
    act = np.ones(2000, bool)
    t = oracle_time(scene, cams, 0, targets, act, "l1")
    r, cores = cpu_fp32_iterations(scene, cams, targets, act, iters=20, sh_degree=0)
    out["plain_2k_64x64_l1"] = {"oracle_s_per_iter": t, "fp32_iters_per_s": r}
    scene, cams, targets = S.workload_fd()
    act = np.ones(500, bool)
    t = oracle_time(scene, cams, 1, targets, act, "l2")
    r, _ = cpu_fp32_iterations(scene, cams, targets, act, iters=20, loss="l2", sh_degree=1)
    out["fd_500_2x32x32_l2"] = {"oracle_s_per_iter": t, "fp32_iters_per_s": r}
    scene, _, cams, masks, _ = S.workload_local(n=100_000, n_views=8, size=800)
    targets = [S.random_image(c, 90 + j) for j, c in enumerate(cams)]
    act = fx.vote_rule(*fx.votes(scene["means"], cams, masks), len(cams))
    tiles = ostep.active_tiles(scene, cams, act)
    t = oracle_time(scene, cams, 3, targets, act, "l1", tiles=tiles)
    r, _ = cpu_fp32_iterations(scene, cams, targets, act, iters=30)
    out["local_100k_8x800"] = {"oracle_s_per_iter": t,
                               "oracle_note": "one iteration over the tiles O^t touches",
                               "fp32_iters_per_s": r, "fp32_note": "30 iterations",
                               "active_gaussians": int(act.sum()),
                               "active_tiles": int(sum(len(x) for x in tiles))}
    return {"cpu_configs": out, "oracle_cores": 1, "fp32_cores": cores,
            "host_cpu_count": os.cpu_count()}


def run_reference(args, rank, world):
    """The CPU oracle on the machine's host cores, each step a bounded sample."""
    import torch
    from oracle import fp32_index as fx
    scene, target_scene, cams, masks, box = setup_workload(args, seed=0)
    c, o = fx.votes(scene["means"], cams, masks)
    active = fx.vote_rule(c, o, len(cams))
    from paper_2506_21117_gb300 import synthetic as S
    targets = [S.random_image(cam, 0) for cam in cams]
    times = []
    cache = {}
    for k in range(args.warmup + args.steps):
        sec, desc = oracle_sample(scene, cams, targets, active, seed=k, cache=cache)
        if k >= args.warmup:
            times.append(sec)
    sec = sum(times) / len(times)
    v = 1.0 / sec
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1,
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.cpu_configs:
        if rank == 0:
            print(json.dumps(run_cpu_configs(args)))
        return 0
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args, rank, world)))
        return 0
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    line = run_ours(args, rank, world)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
