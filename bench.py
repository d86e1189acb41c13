#!/usr/bin/env python
"""Benchmark of the CT augmentation hot path on B300.

One step = one pass of the batched forward augmentation (affine map,
trilinear image + nearest label, intensity affine, Philox noise) over the
64-volume uneven batch: 64 float32 phantoms (in-plane U{96..160}, slices
U{80..240}) warped into 64 crops of 120x120x160 (float32 image + uint8 label)
in ONE persistent launch captured in a CUDA graph.  `value` is output voxels
per second over all ranks (Gvox/s).  Each rank augments its own batch
(weak scaling; no data-path collective).

Also reported on the same line:
  fwd_bwd   -- forward + adjoint (input and affine) on 8 x 128^3 (Gvox/s);
  plain_fwd -- the same 64-volume batch as 64 one-volume launches;
  roofline  -- algorithmic bytes / kernel time vs the measured HBM copy peak;
  e2e       -- the same step through the C ABI from pinned host buffers
               (H2D of inputs, D2H of outputs inside the timed region);
  cpu_baseline -- the FP64 oracle on a bounded sample, single thread.
  iou       -- the fused label warp + IOU loss on 8 x 120x120x160 (Gvox/s);
  train_step -- the full-resolution int16 training step: 16 volumes of
               512^2 x 300-600 -> 128x128x160 crops, forward + IOU + affine
               adjoint in one graph (Gvox/s).
Each of fwd_bwd, iou and train_step carries its own HBM roofline object;
their kernel variants are autotuned on their own workloads (the headline
forward runs the library's default variant unless --variant or --autotune;
--variant also fixes the forward of fwd_bwd).
With --all: the single small volume, the loss variants, the training step
from volumes resampled once to 3 mm, and the anti-aliasing Gaussian.

--impl reference times the FP64 oracle (the only reference implementation
of this method here) on the host cores, on a bounded sample per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "augmented output Gvoxels/s and % of HBM peak; warp fwd+bwd Gvox/s, same tolerance"
WORKLOAD = ("batched 64 uneven f32 volumes (96-160^2 x 80-240) + u8 labels -> "
            "64 x 120x120x160 f32 crops + u8 labels, one persistent launch in a CUDA graph")
FALLBACK_HBM_GBS = 6400.0


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---- peaks, clocks, profile summaries ---------------------------------------------------
def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# Device sources of the forward kernel (its code and its grid cap): a recorded
# DRAM-traffic figure is only used while these are unchanged.
FWD_SOURCES = ("fwd.cu", "fwd.cuh", "common.cuh", "sample.cuh", "sched.cuh")


def kernel_source_hash():
    h = hashlib.sha256()
    for name in FWD_SOURCES:
        with open(os.path.join(ROOT, "paper_1811_11226_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profile_record(name, key, variant=None):
    """A per-launch figure recorded in profiles/<name>.md from an ncu capture
    ('<key>: N' beside 'csrc_hash: H' and 'variant: V'); None if absent, if the
    kernel's sources changed since the capture, or if the capture was of
    another kernel variant than the one timed."""
    p = os.path.join(ROOT, "profiles", f"{name}.md")
    if not os.path.exists(p):
        return None
    kv = {}
    for line in open(p):
        line = line.strip().lstrip("-* ")
        if ":" in line and line.startswith((key, "csrc_hash", "variant")):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip().strip("`")
    if kv.get("csrc_hash") != kernel_source_hash() or key not in kv:
        return None
    if variant is not None and kv.get("variant") != variant:
        return None
    return float(kv[key])


def profile_traffic(name, variant=None):
    """DRAM bytes per launch of the recorded capture (see profile_record)."""
    return profile_record(name, "dram_bytes_per_launch", variant)


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the GPU is busy."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,"
         "utilization.gpu")

    def __init__(self, gpu_index):
        self.proc = None
        self.lines = []
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "20", "-i", str(gpu_index)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 10:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5], f[6], f[7], f[8], float(f[9])))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        busy = [r for r in rows if r[6] > 0] or rows
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in busy:
            for n, v in zip(names, r[2:6]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(r[0] for r in busy),
                "sm_max_mhz": max(r[1] for r in busy), "reasons": sorted(reasons),
                "samples": len(busy)}


# ---- algorithmic bytes --------------------------------------------------------------------
def distinct_refs(v, trilinear=True, device="cuda"):
    """Number of distinct in-volume input elements referenced by the warp of
    one volume (8 trilinear taps, or the nearest voxel), from exact FP64
    coordinates.  Measurement only."""
    onx, ony, onz = v.out_shape
    nz, ny, nx = (int(s) for s in (v.image if v.image is not None else v.label).shape)
    T = torch.tensor(np.asarray(v.T, np.float64), device=device)
    mark = torch.zeros(nx * ny * nz, dtype=torch.bool, device=device)
    i = torch.arange(onx, device=device, dtype=torch.float64)
    j = torch.arange(ony, device=device, dtype=torch.float64)
    step = max(1, (1 << 22) // (onx * ony))
    for k0 in range(0, onz, step):
        k = torch.arange(k0, min(onz, k0 + step), device=device, dtype=torch.float64)
        s = [T[r, 0] * i[None, None, :] + T[r, 1] * j[None, :, None] + T[r, 2] * k[:, None, None]
             + T[r, 3] for r in range(3)]
        if trilinear:
            f = [torch.floor(x).to(torch.int64) for x in s]
            offs = [(dx, dy, dz) for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)]
        else:
            f = [torch.floor(x + 0.5).to(torch.int64) for x in s]
            offs = [(0, 0, 0)]
        for dx, dy, dz in offs:
            x, y, z = f[0] + dx, f[1] + dy, f[2] + dz
            ok = (x >= 0) & (x < nx) & (y >= 0) & (y < ny) & (z >= 0) & (z < nz)
            mark[((z * ny + y) * nx + x)[ok]] = True
    return int(mark.sum().item())


# ---- timing helpers -------------------------------------------------------------------------
def time_graph(graph, steps, warmup, stream):
    """Mean ms per replay of `graph` over exactly `steps` replays on `stream`
    (CUDA events on that stream, barrier + synchronize on both sides)."""
    from paper_1811_11226_b300 import dist as D
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            graph.replay()
        torch.cuda.synchronize()
        D.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            graph.replay()
        e1.record(stream)
        e1.synchronize()
    torch.cuda.synchronize()
    D.barrier()
    return e0.elapsed_time(e1) / steps


def capture(fn, stream):
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        fn()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=stream):
            fn()
    torch.cuda.synchronize()
    return g


# ---- workloads ------------------------------------------------------------------------------
def build_fwd(w, A):
    """Pack a forward workload into contiguous device buffers (so the end-to-end
    leg can move all inputs/outputs with one copy each)."""
    vols = w.vols
    in_sizes = [v.image.numel() for v in vols]
    out_sizes = [v.n_out for v in vols]
    img_all = torch.empty(sum(in_sizes), dtype=vols[0].image.dtype, device="cuda")
    lab_all = torch.empty(sum(in_sizes), dtype=torch.uint8, device="cuda")
    oi_all = torch.empty(sum(out_sizes), dtype=torch.float32, device="cuda")
    ol_all = torch.empty(sum(out_sizes), dtype=torch.uint8, device="cuda")
    imgs, labs, ois, ols = [], [], [], []
    a = b = 0
    for v, ni, no in zip(vols, in_sizes, out_sizes):
        imgs.append(img_all[a:a + ni].view(v.image.shape))
        imgs[-1].copy_(v.image)
        labs.append(lab_all[a:a + ni].view(v.label.shape))
        labs[-1].copy_(v.label)
        onx, ony, onz = v.out_shape
        ois.append(oi_all[b:b + no].view(onz, ony, onx))
        ols.append(ol_all[b:b + no].view(onz, ony, onx))
        a += ni
        b += no
    batch = A.VolumeBatch(imgs, np.stack([v.T for v in vols]), [v.out_shape for v in vols],
                          labels=labs, out_images=ois, out_labels=ols,
                          photo_a=[v.photo_a for v in vols], photo_b=[v.photo_b for v in vols],
                          noise_sigma=[v.sigma for v in vols],
                          noise_ids=[v.noise_id for v in vols])
    return batch, (img_all, lab_all), (oi_all, ol_all)


def fwd_alg_bytes(w):
    tot = 0
    for v in w.vols:
        tot += v.n_out * (4 + 1)
        tot += distinct_refs(v, True) * v.image.element_size()
        tot += distinct_refs(v, False) * 1
    return tot


def run_ours(args, rank, world, local):
    from paper_1811_11226_b300 import augwarp as A
    from paper_1811_11226_b300 import dist as D
    from synth import workloads

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream()
    seed = 0x5EED0000 + rank
    peak, peak_kind = hbm_peak()
    res = {}

    if args.only in ("all", "fwd"):
        # ---- headline: batched forward, 64 uneven volumes ----------------------------------
        w1 = workloads.config1(device=dev)
        for v, nid in zip(w1.vols, D.replica_noise_ids(len(w1.vols), rank)):
            v.noise_id = nid
        batch, (img_all, lab_all), (oi_all, ol_all) = build_fwd(w1, A)
        ws = A.make_workspace(batch.n, 6, dev)
        n_out = sum(batch.out_voxels())
        alg = fwd_alg_bytes(w1)
        fixed = variant_index(A, A.OP_FWD, args.variant)
        if fixed >= 0:
            A.aug_set_variant(A.OP_FWD, fixed)
            best = fixed
        elif args.autotune:
            with torch.cuda.stream(stream):
                best, _ = A.aug_autotune(A.OP_FWD, batch, ws, seed=seed, reps=3)
        else:
            # The library's default variant: the kernel the DRAM-traffic record
            # in profiles/ was captured on.
            best = A.aug_get_variant(A.OP_FWD)
        variant = A.aug_variant_name(A.OP_FWD, best)
        graph = capture(lambda: A.aug_warp_fwd(batch.d_descs, batch.n, seed, ws), stream)
        # Pre-roll at load so the clock samples see the steady state.
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")
        sampler = ClockSampler(vis[local].strip() if len(vis) > local and vis[local].strip()
                               else local)
        t_end = time.time() + (0.0 if args.no_preroll else 1.0)
        with torch.cuda.stream(stream):
            while time.time() < t_end:
                for _ in range(50):
                    graph.replay()
                torch.cuda.synchronize()
        ms = time_graph(graph, args.steps, args.warmup, stream)
        clocks = sampler.stop()
        st, bad = A.aug_read_device_status(ws)
        if st != 0:
            raise RuntimeError(f"device status {A.status_string(st)} volume {bad}")
        ms_max = D.reduce_max(ms, dev if world > 1 else "cpu")
        value = world * n_out / (ms_max * 1e-3) / 1e9
        achieved = alg / (ms * 1e-3) / 1e9
        res.update(value=value, ms=ms_max, n_out=n_out, alg=alg, achieved=achieved, variant=variant,
                   clocks=clocks)
        log(f"[fwd] {variant}: {ms:.4f} ms/step, {n_out / ms / 1e6:.1f} Gvox/s, "
            f"{achieved:.0f} GB/s algorithmic ({alg / 1e9:.3f} GB/step)")

    if args.only == "all":
        # ---- plain one-volume-per-launch forward on the same batch (the 64 launches
        # captured in one graph, so that host launch overhead is not timed) ---------------
        def plain():
            for b in range(batch.n):
                A.aug_warp_fwd_volume(batch.h_descs[b:b + 1], seed)
        g_plain = capture(plain, stream)
        ms_plain = time_graph(g_plain, max(3, min(args.steps, 50)), args.warmup, stream)
        del g_plain
        res["plain"] = {"value": round(n_out / (ms_plain * 1e-3) / 1e9, 3), "unit": "Gvox/s",
                        "ms_per_step": round(ms_plain, 4), "launches_per_step": batch.n}
        log(f"[plain] {ms_plain:.4f} ms/step")

        # ---- the hardware-texture alternative (tex3D linear filtering), same batch ------------
        # A measured comparison only: its interpolation error is several HU (see the tests).
        tw = A.TexWarp(batch.h_descs)
        g_tex = capture(lambda: tw.run(seed), stream)
        ms_tex = time_graph(g_tex, max(3, min(args.steps, 50)), args.warmup, stream)
        del g_tex
        tw.close()
        res["tex3d"] = {"value": round(n_out / (ms_tex * 1e-3) / 1e9, 3), "unit": "Gvox/s",
                        "ms_per_step": round(ms_tex, 4), "launches_per_step": batch.n,
                        "note": "tex3D linear filtering on float32 coordinates, one launch per "
                                "volume; not a parity path (error several HU)"}
        log(f"[tex3d] {ms_tex:.4f} ms/step")

        # ---- end to end through the C ABI from pinned host buffers: aug_warp_fwd_host
        # copies each chunk of volumes in, augments it and copies it out, overlapping
        # the chunks (the host <-> device FIFO of Sec. 4) ---------------------------------
        h_img = torch.empty(img_all.shape, dtype=img_all.dtype, pin_memory=True)
        h_lab = torch.empty(lab_all.shape, dtype=torch.uint8, pin_memory=True)
        h_img.copy_(img_all)
        h_lab.copy_(lab_all)
        h_oi = torch.empty(oi_all.shape, dtype=torch.float32, pin_memory=True)
        h_ol = torch.empty(ol_all.shape, dtype=torch.uint8, pin_memory=True)
        hv_img, hv_lab, hv_oi, hv_ol = [], [], [], []
        a = b = 0
        for v in w1.vols:
            ni, no = v.image.numel(), v.n_out
            onx, ony, onz = v.out_shape
            hv_img.append(h_img[a:a + ni].view(v.image.shape))
            hv_lab.append(h_lab[a:a + ni].view(v.image.shape))
            hv_oi.append(h_oi[b:b + no].view(onz, ony, onx))
            hv_ol.append(h_ol[b:b + no].view(onz, ony, onx))
            a += ni
            b += no
        h_descs = A.host_descriptors(hv_img, np.stack([v.T for v in w1.vols]),
                                     [v.out_shape for v in w1.vols], labels=hv_lab,
                                     out_images=hv_oi, out_labels=hv_ol,
                                     photo_a=[v.photo_a for v in w1.vols],
                                     photo_b=[v.photo_b for v in w1.vols],
                                     noise_sigma=[v.sigma for v in w1.vols],
                                     noise_ids=[v.noise_id for v in w1.vols])

        def time_e2e(chunk, k):
            with torch.cuda.stream(stream):
                for _ in range(2):
                    A.aug_warp_fwd_host(h_descs, seed, chunk)
                torch.cuda.synchronize()
                D.barrier()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(k):
                    A.aug_warp_fwd_host(h_descs, seed, chunk)
                e1.record(stream)
                e1.synchronize()
            return D.reduce_max(e0.elapsed_time(e1) / k, dev if world > 1 else "cpu")
        k_e2e = max(3, min(args.steps, 20))
        ms_e2e = time_e2e(8, k_e2e)
        ms_seq = time_e2e(batch.n, max(3, k_e2e // 2))

        # Copy bound of this box: the same bytes moved both ways at once, no compute.
        s_up, s_dn = torch.cuda.Stream(), torch.cuda.Stream()

        def copies():
            s_up.wait_stream(stream)
            s_dn.wait_stream(stream)
            with torch.cuda.stream(s_up):
                img_all.copy_(h_img, non_blocking=True)
                lab_all.copy_(h_lab, non_blocking=True)
            with torch.cuda.stream(s_dn):
                h_oi.copy_(oi_all, non_blocking=True)
                h_ol.copy_(ol_all, non_blocking=True)
            stream.wait_stream(s_up)
            stream.wait_stream(s_dn)
        with torch.cuda.stream(stream):
            copies()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(5):
                copies()
            e1.record(stream)
            e1.synchronize()
        ms_copy = e0.elapsed_time(e1) / 5
        # the host outputs are the device path's
        A.aug_warp_fwd_host(h_descs, seed, 8)
        torch.cuda.synchronize()
        A.aug_warp_fwd(batch.d_descs, batch.n, seed, ws)
        if not torch.equal(h_oi, oi_all.cpu()) or not torch.equal(h_ol, ol_all.cpu()):
            raise RuntimeError("host-buffer forward differs from the device forward")
        res["e2e"] = {"value": round(world * n_out / (ms_e2e * 1e-3) / 1e9, 3), "unit": "Gvox/s",
                      "h2d_bytes_per_step": int(img_all.numel() * img_all.element_size() +
                                                lab_all.numel()),
                      "d2h_bytes_per_step": int(oi_all.numel() * 4 + ol_all.numel()),
                      "ms_per_step": round(ms_e2e, 3), "steps": k_e2e,
                      "api": "aug_warp_fwd_host, chunks of 8 volumes on 3 streams",
                      "single_chunk_ms": round(ms_seq, 3),
                      "copy_bound_ms": round(ms_copy, 3),
                      "frac_of_copy_bound": round(ms_copy / ms_e2e, 4)}
        log(f"[e2e] {ms_e2e:.3f} ms/step pipelined, {ms_seq:.3f} ms/step as one chunk, "
            f"copies alone (both directions at once) {ms_copy:.3f} ms")
        del h_img, h_lab, h_oi, h_ol

    if args.only == "all":
        # ---- forward with the parameters drawn on the device (same ranges as the host
        # draw of the batch: rotation +-15 deg, scale 0.9-1.1, shift +-10, a 0.9-1.1,
        # b +-50, sigma 0-50), sampler + forward in one graph, new draw every replay ----
        d_descs2 = batch.d_descs.clone()
        spec = A.ParamSpec(rot_max=(np.deg2rad(15.0),) * 3, scale_min=(0.9,) * 3,
                           scale_max=(1.1,) * 3, shift_max=(10.0,) * 3, photo_a=(0.9, 1.1),
                           photo_b=(-50.0, 50.0), sigma=(0.0, 50.0),
                           draw=A.AUG_DRAW_AFFINE | A.AUG_DRAW_PHOTO)
        counter = torch.zeros(1, dtype=torch.int64, device=dev)

        def sampled_step():
            A.aug_sample_params(d_descs2, batch.n, spec, seed, counter=counter)
            A.aug_warp_fwd(d_descs2, batch.n, seed, ws)
        g2 = capture(sampled_step, stream)
        ms_s = time_graph(g2, max(3, args.steps // 5), args.warmup, stream)
        st, bad = A.aug_read_device_status(ws)
        if st != 0:
            raise RuntimeError(f"device status {A.status_string(st)} volume {bad}")
        res["fwd_device_params"] = {
            "value": round(world * n_out / (ms_s * 1e-3) / 1e9, 3), "unit": "Gvox/s",
            "ms_per_step": round(ms_s, 4), "draws": int(counter.item()),
            "workload": "same batch, affine + intensity drawn per volume on the device "
                        "(aug_sample_params) inside the graph"}
        log(f"[fwd+device params] {ms_s:.4f} ms/step")

    # ---- forward + backward, 8 x 128^3 --------------------------------------------------------
    if args.only in ("all", "fwd_bwd"):
        res["fwd_bwd"] = bench_fwd_bwd(args, A, D, dev, stream, seed, world)
    if args.only == "all" and args.all:
        res["config0"] = bench_config0(args, A, dev, stream, seed)
    if args.only in ("all", "iou"):
        res["iou"] = bench_iou(args, A, dev, stream)
    if (args.only == "all" and args.all) or args.only == "loss":
        res["loss_variants"] = bench_loss_variants(args, A, dev, stream)
    if args.only in ("all", "train"):
        res["train_step"] = bench_train(args, A, dev, stream, seed)
    if (args.only == "all" and args.all) or args.only == "train":
        res["train_step_resampled"] = bench_train_resampled(args, A, dev, stream, seed)
    if (args.only == "all" and args.all) or args.only == "smooth":
        res["antialias_smooth"] = bench_smooth(args, A, dev, stream)
    res["peak"], res["peak_kind"] = peak, peak_kind
    # Each graph replay of the headline step launches two of the library's
    # kernels: the descriptor prologue (k_prepare) and the forward (k_fwd_batched or
    # k_fwd_batched_box, by variant).
    res["launches"] = 2 * args.steps
    return res


def bench_fwd_bwd(args, A, D, dev, stream, seed, world):
    from synth import workloads
    w = workloads.config2(device=dev)
    vols = w.vols
    out = [torch.empty(tuple(reversed(v.out_shape)), device=dev) for v in vols]
    batch = A.VolumeBatch([v.image for v in vols], np.stack([v.T for v in vols]),
                          [v.out_shape for v in vols], out_images=out,
                          noise_ids=[v.noise_id for v in vols])
    gptr = A.pointer_array(w.g, dev)
    gin = [torch.empty_like(v.image) for v in vols]
    giptr = A.pointer_array(gin, dev)
    gaff = torch.empty((len(vols), 3, 4), device=dev)
    ws = A.make_workspace(len(vols), 0, dev)
    # The step's forward kernel is autotuned on this workload too (the
    # previous choice is restored afterwards), unless a variant is fixed.
    fwd_prev = A.aug_get_variant(A.OP_FWD)
    if variant_index(A, A.OP_FWD, args.variant) < 0:
        with torch.cuda.stream(stream):
            A.aug_autotune(A.OP_FWD, batch, ws, seed=seed, reps=3)
    if variant_index(A, A.OP_BWD, args.bwd_variant) >= 0:
        A.aug_set_variant(A.OP_BWD, variant_index(A, A.OP_BWD, args.bwd_variant))
    else:
        with torch.cuda.stream(stream):
            A.aug_autotune(A.OP_BWD, batch, ws, grad_out_ptrs=gptr, grad_in_ptrs=giptr,
                           grad_affine=gaff, reps=3)
    fwd_variant = A.aug_variant_name(A.OP_FWD, A.aug_get_variant(A.OP_FWD))

    def step():
        A.aug_warp_fwd(batch.d_descs, batch.n, seed, ws)
        A.aug_warp_bwd(batch.d_descs, batch.n, gptr, giptr, gaff, ws)
    graph = capture(step, stream)
    ms = time_graph(graph, max(3, args.steps // 5), args.warmup, stream)
    A.aug_set_variant(A.OP_FWD, fwd_prev)
    n_out = sum(v.n_out for v in vols)
    alg = 0
    for v in vols:
        foot = distinct_refs(v, True)
        alg += v.n_out * 4 + foot * 4            # forward: taps + image out
        alg += v.n_out * 4 + foot * 4            # adjoint: g + taps
        alg += v.image.numel() * 4               # grad_in written
    ms_max = D.reduce_max(ms, dev if world > 1 else "cpu")
    log(f"[fwd+bwd] {ms:.4f} ms/step")
    return {"value": round(world * n_out / (ms_max * 1e-3) / 1e9, 3), "unit": "Gvox/s",
            "ms_per_step": round(ms_max, 4), "workload": "8 x 128^3 f32, fwd + grad_in + grad_T",
            "alg_GBps": round(alg / (ms * 1e-3) / 1e9, 1),
            "roofline": sub_roofline(alg, ms, "forward + adjoint step (prologue, forward, "
                                     "zeroing, adjoint, finalize)"),
            "variant": A.aug_variant_name(A.OP_BWD, A.aug_get_variant(A.OP_BWD)),
            "fwd_variant": fwd_variant}


def bench_config0(args, A, dev, stream, seed):
    """The single 128x128x64 f32 volume (+ labels) of the smallest configuration:
    its 5 MB of output and input sit in L2, so the step is launch-bound (one
    prologue + one forward launch per graph replay); reported for completeness."""
    from synth import workloads
    w = workloads.config0(device=dev)
    v = w.vols[0]
    onx, ony, onz = v.out_shape
    oi = torch.empty((onz, ony, onx), device=dev)
    ol = torch.empty((onz, ony, onx), dtype=torch.uint8, device=dev)
    batch = A.VolumeBatch([v.image], np.stack([v.T]), [v.out_shape], labels=[v.label],
                          out_images=[oi], out_labels=[ol], photo_a=[v.photo_a],
                          photo_b=[v.photo_b], noise_sigma=[v.sigma], noise_ids=[0])
    ws = A.make_workspace(1, 0, dev)
    graph = capture(lambda: A.aug_warp_fwd(batch.d_descs, 1, seed, ws), stream)
    ms = time_graph(graph, max(20, args.steps), args.warmup, stream)
    log(f"[config0] {ms * 1e3:.1f} us/step")
    return {"value": round(v.n_out / (ms * 1e-3) / 1e9, 3), "unit": "Gvox/s",
            "ms_per_step": round(ms, 5),
            "workload": "1 x 128x128x64 f32 + labels (L2-resident: launch-bound)"}


def bench_iou(args, A, dev, stream):
    from synth import workloads
    w = workloads.config3(device=dev)
    vols = w.vols
    batch = A.VolumeBatch([None] * len(vols), np.stack([v.T for v in vols]),
                          [v.out_shape for v in vols], labels=[v.label for v in vols], device=dev)
    ws = A.make_workspace(len(vols), 6, dev)
    loss = torch.empty(len(vols), device=dev)
    gp = torch.empty_like(w.p)
    if variant_index(A, A.OP_IOU, args.iou_variant) >= 0:
        A.aug_set_variant(A.OP_IOU, variant_index(A, A.OP_IOU, args.iou_variant))
    else:
        with torch.cuda.stream(stream):
            A.aug_autotune(A.OP_IOU, batch, ws, p=w.p, n_classes=6, loss=loss, grad_p=gp,
                           reps=3)
    graph = capture(lambda: A.iou_loss_fwd_bwd(batch.d_descs, batch.n, w.p, 6, loss, gp, ws),
                    stream)
    ms = time_graph(graph, max(3, args.steps // 5), args.warmup, stream)
    n_out = sum(v.n_out for v in vols)
    alg = n_out * 6 * 4 * 2 + sum(distinct_refs(v, False) for v in vols)
    log(f"[iou] {ms:.4f} ms/step")
    return {"value": round(n_out / (ms * 1e-3) / 1e9, 3), "unit": "Gvox/s",
            "ms_per_step": round(ms, 4), "alg_GBps": round(alg / (ms * 1e-3) / 1e9, 1),
            "roofline": sub_roofline(alg, ms, "fused label warp + IOU step (prologue, sums "
                                     "pass, finalize, gradient pass)"),
            "alg_bytes": "p read 24 B + grad_p written 24 B per output voxel + distinct labels",
            "workload": "8 x 120x120x160 label warp + IOU fwd/bwd, 6 classes"}


def bench_loss_variants(args, A, dev, stream):
    """Sec. 5.C loss variants on the 8 x 120x120x160 workload: Dice and the
    p^2 family on probabilities (x read once, grad written), and both with the
    softmax over 6 class scores fused in (scores read by both passes)."""
    from synth import workloads
    w = workloads.config3(device=dev)
    vols = w.vols
    batch = A.VolumeBatch([None] * len(vols), np.stack([v.T for v in vols]),
                          [v.out_shape for v in vols], labels=[v.label for v in vols], device=dev)
    ws = A.make_workspace(len(vols), 6, dev)
    loss = torch.empty(len(vols), device=dev)
    scores = workloads.class_logits([v.out_shape for v in vols], seed=3, device=dev)
    gx = torch.empty_like(w.p)
    n_out = sum(v.n_out for v in vols)
    labs = sum(distinct_refs(v, False) for v in vols)
    out = []
    for name, kind, power, logits in [("dice", A.AUG_LOSS_DICE, 1.0, False),
                                      ("iou_p2", A.AUG_LOSS_IOU, 2.0, False),
                                      ("dice_softmax", A.AUG_LOSS_DICE, 1.0, True),
                                      ("iou_p2_softmax", A.AUG_LOSS_IOU, 2.0, True)]:
        x = scores if logits else w.p
        graph = capture(lambda: A.seg_loss_fwd_bwd(batch.d_descs, batch.n, x, 6, loss, gx, ws,
                                                   kind, power, logits), stream)
        ms = time_graph(graph, max(3, args.steps // 5), args.warmup, stream)
        reads = 1 if (kind == A.AUG_LOSS_DICE and power == 1.0 and not logits) else 2
        alg = n_out * 6 * 4 * (reads + 1) + labs
        log(f"[loss {name}] {ms:.4f} ms/step")
        out.append({"loss": name, "value": round(n_out / (ms * 1e-3) / 1e9, 3), "unit": "Gvox/s",
                    "ms_per_step": round(ms, 4), "alg_GBps": round(alg / (ms * 1e-3) / 1e9, 1)})
    return out


def tune_step_kernels(A, batch, ws, seed, p, loss, gp, gptr, gaff, stream):
    """Autotunes the forward, loss and affine-adjoint kernels of a training step
    on its own workload (as the forward + adjoint and IOU legs do on theirs);
    returns the chosen variant names and the previous variants, to restore."""
    ops = (A.OP_FWD, A.OP_IOU, A.OP_BWD)
    prev = [A.aug_get_variant(op) for op in ops]
    with torch.cuda.stream(stream):
        A.aug_autotune(A.OP_FWD, batch, ws, seed=seed, reps=3)
        A.aug_autotune(A.OP_IOU, batch, ws, p=p, n_classes=6, loss=loss, grad_p=gp, reps=3)
        A.aug_autotune(A.OP_BWD, batch, ws, grad_out_ptrs=gptr, grad_affine=gaff, reps=3)
    torch.cuda.synchronize()
    names = {k: A.aug_variant_name(op, A.aug_get_variant(op))
             for k, op in zip(("fwd", "loss", "adjoint"), ops)}
    return names, list(zip(ops, prev))


def restore_variants(A, saved):
    for op, v in saved:
        A.aug_set_variant(op, v)


def bench_train(args, A, dev, stream, seed):
    from synth import workloads
    w = workloads.config4(device=dev, n_vols=args.train_vols)
    vols = w.vols
    out = [torch.empty(tuple(reversed(v.out_shape)), device=dev) for v in vols]
    batch = A.VolumeBatch([v.image for v in vols], np.stack([v.T for v in vols]),
                          [v.out_shape for v in vols], labels=[v.label for v in vols],
                          out_images=out, photo_a=[v.photo_a for v in vols],
                          photo_b=[v.photo_b for v in vols], noise_sigma=[v.sigma for v in vols],
                          noise_ids=[v.noise_id for v in vols])
    ws = A.make_workspace(len(vols), 6, dev)
    loss = torch.empty(len(vols), device=dev)
    gp = torch.empty_like(w.p)
    gptr = A.pointer_array(w.g, dev)
    gaff = torch.empty((len(vols), 3, 4), device=dev)

    variants, saved = tune_step_kernels(A, batch, ws, seed, w.p, loss, gp, gptr, gaff, stream)

    def step():
        A.aug_warp_fwd(batch.d_descs, batch.n, seed, ws)
        A.iou_loss_fwd_bwd(batch.d_descs, batch.n, w.p, 6, loss, gp, ws)
        A.aug_warp_bwd(batch.d_descs, batch.n, gptr, None, gaff, ws)
    graph = capture(step, stream)
    ms = time_graph(graph, max(3, args.steps // 10), args.warmup, stream)
    restore_variants(A, saved)
    n_out = sum(v.n_out for v in vols)
    alg = 0
    for v in vols:
        foot = distinct_refs(v, True)
        labs = distinct_refs(v, False)
        alg += foot * 2 + v.n_out * 4            # forward image
        alg += v.n_out * 48 + labs               # IOU: p read, grad_p write, labels
        alg += v.n_out * 4 + foot * 2            # affine adjoint: g + taps
    log(f"[train] {ms:.4f} ms/step")
    return {"value": round(n_out / (ms * 1e-3) / 1e9, 3), "unit": "Gvox/s",
            "ms_per_step": round(ms, 4), "alg_GBps": round(alg / (ms * 1e-3) / 1e9, 1),
            "roofline": sub_roofline(alg, ms, "training step (forward, IOU fwd/bwd, affine "
                                     "adjoint) in one graph"),
            "workload": f"{len(vols)} int16 512^2 x 300-600 -> 128x128x160: fwd + IOU fwd/bwd + "
                        "grad_T",
            "variants": {**variants, "chosen": "autotuned on this workload"}}


def bench_train_resampled(args, A, dev, stream, seed):
    """The paper's order for the full-resolution volumes: resample once to 3 mm
    (anti-aliasing Gaussian, then the 3/0.7 downscaling warp of image and
    labels), then run the same training step (forward + loss + affine adjoint
    to 128x128x160 crops) from the small volumes.  Reports the one-time
    resampling and the per-step time."""
    from synth import workloads
    from synth.params import AffineSpec, random_affine
    w = workloads.config4(device=dev, n_vols=args.train_vols)
    down = 3.0 / 0.7
    s = A.aug_antialias_sigma(3.0, 0.7)
    imgs = [v.image for v in w.vols]
    sm = [torch.empty(im.shape, device=dev) for im in imgs]
    small_i, small_l, descs = [], [], []
    for v in w.vols:
        nz, ny, nx = v.image.shape
        sx, sy, sz = (max(1, int(round(n / down))) for n in (nx, ny, nz))
        small_i.append(torch.empty((sz, sy, sx), device=dev))
        small_l.append(torch.empty((sz, sy, sx), dtype=torch.uint8, device=dev))
        T = np.zeros((3, 4), np.float32)
        for r, (n_in, n_out) in enumerate(((nx, sx), (ny, sy), (nz, sz))):
            T[r, r] = down
            T[r, 3] = (n_in - 1) / 2.0 - down * (n_out - 1) / 2.0
        descs.append(T)
    rs = A.VolumeBatch(sm, np.stack(descs), [tuple(reversed(t.shape)) for t in small_i],
                       labels=[v.label for v in w.vols], out_images=small_i, out_labels=small_l,
                       device=dev)
    rs_ws = A.make_workspace(len(w.vols), 0, dev)

    def resample():
        A.aug_smooth(imgs, sm, [(s, s, s)] * len(imgs))
        A.aug_warp_fwd(rs.d_descs, rs.n, 0, rs_ws)
    g0 = capture(resample, stream)
    ms_rs = time_graph(g0, 3, 1, stream)

    # The training step from the resampled volumes: random augmentation affines
    # (rotation, scale, shift) to 128x128x160 crops, photometric draw as before.
    rng = np.random.default_rng(44)
    out = [torch.empty((160, 128, 128), device=dev) for _ in w.vols]
    Ts = [random_affine(rng, tuple(reversed(t.shape)), (128, 128, 160), AffineSpec())[0]
          for t in small_i]
    batch = A.VolumeBatch(small_i, np.stack(Ts), [(128, 128, 160)] * len(w.vols),
                          labels=small_l, out_images=out, photo_a=[v.photo_a for v in w.vols],
                          photo_b=[v.photo_b for v in w.vols],
                          noise_sigma=[v.sigma for v in w.vols],
                          noise_ids=[v.noise_id for v in w.vols])
    ws = A.make_workspace(len(w.vols), 6, dev)
    loss = torch.empty(len(w.vols), device=dev)
    gp = torch.empty_like(w.p)
    gptr = A.pointer_array(w.g, dev)
    gaff = torch.empty((len(w.vols), 3, 4), device=dev)
    variants, saved = tune_step_kernels(A, batch, ws, seed, w.p, loss, gp, gptr, gaff, stream)

    def step():
        A.aug_warp_fwd(batch.d_descs, batch.n, seed, ws)
        A.iou_loss_fwd_bwd(batch.d_descs, batch.n, w.p, 6, loss, gp, ws)
        A.aug_warp_bwd(batch.d_descs, batch.n, gptr, None, gaff, ws)
    graph = capture(step, stream)
    ms = time_graph(graph, max(3, args.steps // 10), args.warmup, stream)
    restore_variants(A, saved)
    st, bad = A.aug_read_device_status(ws)
    if st != 0 or A.aug_read_device_status(rs_ws)[0] != 0 or A.aug_smooth_status() != 0:
        raise RuntimeError("device status after the resampled training step")
    n_out = sum(v.n_out for v in w.vols)
    log(f"[train resampled] {ms:.4f} ms/step (one-time resampling {ms_rs:.3f} ms)")
    return {"value": round(n_out / (ms * 1e-3) / 1e9, 3), "unit": "Gvox/s",
            "ms_per_step": round(ms, 4), "one_time_resampling_ms": round(ms_rs, 3),
            "workload": f"{len(w.vols)} int16 512^2 x 300-600 resampled once to 3 mm "
                        "(smooth + downscale), then fwd + IOU fwd/bwd + grad_T to 128x128x160",
            "variants": {**variants, "chosen": "autotuned on this workload"}}


def bench_smooth(args, A, dev, stream):
    """Anti-aliasing Gaussian of the 3 mm resampling (Sec. 5.A) on the 16
    full-resolution int16 volumes (512^2 x 300-600, 0.7 mm -> 3 mm:
    sigma = (3/0.7 - 1)/3 = 1.095 voxels, 9 taps per axis): int16 in, float32
    out, HBM-bound at 6 bytes per voxel."""
    from synth import workloads
    w = workloads.config4(device=dev, n_vols=args.smooth_vols)
    imgs = [v.image for v in w.vols]
    outs = [torch.empty(im.shape, dtype=torch.float32, device=dev) for im in imgs]
    s = A.aug_antialias_sigma(3.0, 0.7)
    graph = capture(lambda: A.aug_smooth(imgs, outs, [(s, s, s)] * len(imgs)), stream)
    ms = time_graph(graph, max(3, args.steps // 20), args.warmup, stream)
    nvox = sum(im.numel() for im in imgs)
    alg = nvox * (2 + 4)
    peak, _ = hbm_peak()
    log(f"[smooth] {ms:.4f} ms/step")
    return {"value": round(nvox / (ms * 1e-3) / 1e9, 3), "unit": "Gvox/s (input voxels)",
            "ms_per_step": round(ms, 4), "alg_GBps": round(alg / (ms * 1e-3) / 1e9, 1),
            "frac_of_hbm": round(alg / (ms * 1e-3) / 1e9 / peak, 4),
            "workload": f"{len(imgs)} int16 512^2 x 300-600 -> float32, sigma 1.095 "
                        "(9 taps per axis)"}


# ---- CPU baseline: the FP64 oracle ----------------------------------------------------------
def cpu_baseline(min_seconds=15.0):
    from oracle import ref
    from synth import workloads
    # Inputs are generated on the GPU (fast) and copied to the host per volume.
    w = workloads.config1(device="cuda" if torch.cuda.is_available() else "cpu")
    done, t0 = 0, time.perf_counter()
    nv = 0
    for v in w.vols:
        ref.warp_fwd(v, 1)
        done += v.n_out
        nv += 1
        if time.perf_counter() - t0 >= min_seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": round(done / dt / 1e9, 6), "unit": "Gvox/s", "cores": 1, "kind": "oracle",
            "sample": f"first {nv} volumes of the 64-volume batch ({done / 1e6:.1f} Mvox), "
                      f"full forward (image + label + noise), FP64, single thread, {dt:.1f} s"}


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores: each step evaluates a fixed sample of
    output voxels of the 64-volume batch, split over all cores."""
    if rank != 0:
        return None
    import concurrent.futures as cfut
    from oracle import ref
    from synth import workloads
    cores = os.cpu_count() or 1
    w = workloads.config1(device="cpu")
    rng = np.random.default_rng(0)
    per_thread = 8192
    # One contiguous run of output voxels per thread per step, cycling over volumes.
    jobs = []
    for s in range(args.warmup + args.steps):
        step = []
        for t in range(cores):
            b = (s * cores + t) % len(w.vols)
            v = w.vols[b]
            q0 = int(rng.integers(0, v.n_out - per_thread))
            step.append((b, np.arange(q0, q0 + per_thread, dtype=np.int64)))
        jobs.append(step)
    pool = cfut.ThreadPoolExecutor(max_workers=cores)
    run = lambda job: ref.warp_fwd_points(w.vols[job[0]], 1, job[1])
    for s in range(args.warmup):
        list(pool.map(run, jobs[s]))
    t0 = time.perf_counter()
    for s in range(args.warmup, args.warmup + args.steps):
        list(pool.map(run, jobs[s]))
    dt = time.perf_counter() - t0
    pool.shutdown()
    n = cores * per_thread * args.steps
    value = n / dt / 1e9
    return {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "Gvox/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "global_batch": 64, "per_step_sample":
                       f"{cores} x {per_thread} output voxels"},
            "cpu_baseline": {"value": round(value, 6), "unit": "Gvox/s", "cores": cores,
                             "kind": "oracle",
                             "sample": f"{cores} threads x {per_thread} contiguous output voxels "
                                       "per step (forward: image + label + noise, FP64)"},
            "e2e": {"value": round(value, 6), "unit": "Gvox/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def variant_index(A, op, spec) -> int:
    """Index of a kernel variant given as an index or a name (-1: none fixed)."""
    spec = str(spec)
    if spec.lstrip("-").isdigit():
        return int(spec)
    for v in range(A.aug_num_variants(op)):
        if A.aug_variant_name(op, v) == spec:
            return v
    raise SystemExit(f"unknown variant {spec!r} of op {op}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--all", action="store_true", help="also time the IOU and training-step "
                    "workloads")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only", choices=["all", "fwd", "fwd_bwd", "iou", "loss", "train", "smooth"],
                    default="all", help="time one workload only (profiling runs)")
    ap.add_argument("--variant", default="-1",
                    help="fixed forward kernel variant, by index or name (default: the "
                         "library's default)")
    ap.add_argument("--iou-variant", default="-1",
                    help="fixed loss kernel variant, by index or name (default: autotuned on "
                         "the workload)")
    ap.add_argument("--bwd-variant", default="-1",
                    help="fixed adjoint kernel variant, by index or name (default: autotuned "
                         "on the workload)")
    ap.add_argument("--autotune", action="store_true",
                    help="pick the forward variant by timing all of them first")
    ap.add_argument("--no-preroll", action="store_true")
    ap.add_argument("--train-vols", type=int, default=16,
                    help="volumes of the training-step workload (profiling runs use fewer)")
    ap.add_argument("--smooth-vols", type=int, default=16,
                    help="volumes of the smoothing workload (profiling runs use fewer)")
    ap.add_argument("--summarize-ncu", metavar="CSV",
                    help="print the per-kernel summary of an ncu --csv log (and, with "
                         "--kernel, the record lines of profiles/*.md) and exit")
    ap.add_argument("--kernel", help="kernel-name regex for --summarize-ncu")
    ap.add_argument("--record-variant", help="variant name the --summarize-ncu capture ran")
    args = ap.parse_args()
    if args.summarize_ncu:
        summarize_ncu(args.summarize_ncu, args.kernel, variant=args.record_variant)
        return
    args.warmup = max(3, args.warmup)

    from paper_1811_11226_b300 import dist as D
    if args.impl == "reference":
        rank, world, _ = D.env_rank_world()
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return

    rank, world, local = D.init_from_env("nccl")
    res = run_ours(args, rank, world, local)
    if rank != 0:
        return
    if args.only != "all":
        keep = {k: v for k, v in res.items() if k in ("fwd_bwd", "iou", "loss_variants",
                                                       "train_step", "train_step_resampled",
                                                       "antialias_smooth", "ms", "value",
                                                       "variant", "achieved")}
        print(json.dumps({"profile_run": args.only, **keep}), flush=True)
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()
    peak = res["peak"]
    traffic = profile_traffic("fwd_batched_config1", res["variant"])
    line = {
        "metric": METRIC,
        "value": round(res["value"], 3),
        "unit": "Gvox/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(res["ms"], 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": 64 * world,
                   "out_voxels_per_step": res["n_out"] * world,
                   "parallelism": f"{world} independent replicas (volume batches), no collective",
                   "l2": "inputs 857 MB per step > 126 MB L2, no flush",
                   "variant": res["variant"]},
        "roofline": {"bound": "hbm", "achieved": round(res["achieved"], 1), "peak": peak,
                     "unit": "GB/s", "frac": round(res["achieved"] / peak, 4),
                     "peak_kind": peak_kind_note(res["peak_kind"]),
                     "frac_of_nominal_7700": round(res["achieved"] / 7700.0, 4),
                     "traffic": traffic, "alg_bytes_per_launch": res["alg"],
                     "traffic_source": None if traffic is None else (
                         "profiles/fwd_batched_config1.md: dram__bytes_read.sum + "
                         "dram__bytes_write.sum of one ncu capture of this kernel variant, "
                         "record lines printed by bench.py --summarize-ncu from that capture's "
                         f"CSV (csrc_hash {kernel_source_hash()})"),
                     "kernel": fwd_kernel_name(res["variant"])},
        # The forward is limited by instruction issue, not DRAM: its recorded
        # warp instructions per launch over the measured launch time, against
        # 4 schedulers x SMs x the SM clock sampled during the timed region.
        "issue": issue_roofline(res),
        "fwd_bwd": res["fwd_bwd"],
        "fwd_device_params": res.get("fwd_device_params"),
        "plain_fwd": res["plain"],
        "tex3d_alternative": res.get("tex3d"),
        "e2e": res["e2e"],
        "gpu_launches": res["launches"],
        "clocks": res["clocks"],
        "cpu_baseline": cpu,
    }
    for key in ("config0", "iou", "loss_variants", "train_step", "train_step_resampled",
                "antialias_smooth"):
        if key in res:
            line[key] = res[key]
    print(json.dumps(line), flush=True)


def sub_roofline(alg_bytes, ms, what):
    """HBM roofline of a whole step: algorithmic bytes / step time against the
    measured copy peak (the step's kernels together, one graph replay)."""
    peak, kind = hbm_peak()
    achieved = alg_bytes / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_kind": peak_kind_note(kind),
            "alg_bytes_per_step": int(alg_bytes), "over": what}


def summarize_ncu(path, kernel_regex=None, variant=None):
    """Summary of an ncu --csv log (one row per kernel launch and metric):
    per kernel its launches, total and mean gpu__time_duration, and the mean
    per launch of every other metric, plus the record lines that
    profile_record() reads (for the kernel matching kernel_regex)."""
    import csv
    import re
    rows = [r for r in csv.reader(open(path)) if len(r) > 10]
    hdr = rows[0]
    col = {h: i for i, h in enumerate(hdr)}
    per = {}
    for r in rows[1:]:
        if r[col["ID"]] == "ID":
            continue
        name = r[col["Kernel Name"]]
        met, unit = r[col["Metric Name"]], r[col["Metric Unit"]]
        val = float(r[col["Metric Value"]].replace(",", ""))
        scale = {"ns": 1e-6, "us": 1e-3, "usecond": 1e-3, "msecond": 1.0, "ms": 1.0,
                 "nsecond": 1e-6, "byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
        val *= scale.get(unit, 1.0)
        d = per.setdefault(name, {}).setdefault(met, [])
        d.append(val)
    total_t = sum(sum(m.get("gpu__time_duration.sum", [0.0])) for m in per.values())
    out = []
    for name, m in sorted(per.items(), key=lambda kv: -sum(kv[1].get("gpu__time_duration.sum",
                                                                      [0.0]))):
        t = m.get("gpu__time_duration.sum", [])
        line = f"{name[:60]:60s} launches {len(t):5d}  total {sum(t):9.3f} ms  " \
               f"mean {1e3 * sum(t) / max(len(t), 1):9.1f} us  share {sum(t) / total_t:6.1%}" \
            if t else name
        for met, v in m.items():
            if met != "gpu__time_duration.sum":
                line += f"  {met} {sum(v) / len(v):.6g}"
        out.append(line)
    print("\n".join(out))
    if kernel_regex:
        hits = [m for n, m in per.items() if re.search(kernel_regex, n)]
        if len(hits) == 1:
            m = hits[0]
            rd, wr = m.get("dram__bytes_read.sum"), m.get("dram__bytes_write.sum")
            if rd and wr:
                print(f"- dram_bytes_per_launch: {int(round(sum(rd) / len(rd) + sum(wr) / len(wr)))}")
            if m.get("smsp__inst_executed.sum"):
                v = m["smsp__inst_executed.sum"]
                print(f"- warp_inst_per_launch: {int(round(sum(v) / len(v)))}")
            if variant:
                print(f"- variant: {variant}")
            print(f"- csrc_hash: {kernel_source_hash()}")


def fwd_kernel_name(variant):
    """Kernel that a forward variant launches (the variant tables' naming)."""
    if variant.startswith("b8") or variant.startswith("b16") or variant.startswith("b4"):
        return "k_fwd_batched_box"
    if variant.startswith("brick"):
        return "k_fwd_brick"
    if variant.startswith("bulk"):
        return "k_fwd_brick_bulk"
    return "k_fwd_batched"


def issue_roofline(res):
    inst = profile_record("fwd_batched_config1", "warp_inst_per_launch", res["variant"])
    sm_mhz = (res.get("clocks") or {}).get("sm_mhz")
    if inst is None or not sm_mhz:
        return None
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = 4.0 * sms * sm_mhz * 1e6 / 1e9      # G warp instructions / s
    achieved = inst / (res["ms"] * 1e-3) / 1e9
    return {"bound": "issue", "achieved": round(achieved, 1), "peak": round(peak, 1),
            "unit": "G warp inst/s", "frac": round(achieved / peak, 4),
            "warp_inst_per_launch": int(inst), "kernel": fwd_kernel_name(res["variant"])}


def peak_kind_note(kind):
    return "of measured (MEASURED_PEAKS hbm_gbs)" if kind == "measured" else "of fallback"


if __name__ == "__main__":
    main()
