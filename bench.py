"""Benchmark: partitioned time steps of the 64^3 lid-driven cavity (274,625 nodes,
12 unknowns per node) through libfsi, on one GB300 per rank.

A step is one full time step of the method (Section 2.5): predictor, nonlinear
iterations of the NS, Allen-Cahn and B blocks (each a Newton step solved by
Jacobi-preconditioned GMRES(30) to rel-res 1e-8), corrector.  The metric is the
operator-apply throughput sustained inside those solves: the DoFs of every block
residual and Jacobian-vector product the step evaluates, per second (GDoF/s);
seconds per time step are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32ir|fp64]
  python bench.py --impl reference ...   # the FP64 numpy oracle on the host cores

Under torchrun each rank advances its own replica of the cavity (weak scaling, no
data exchange); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "GDoF/s operator apply; s/timestep to rel-res 1e-8: learned-PC vs plain GMRES"
UNIT = "GDoF/s"
WORKLOAD = "cavity64: 3D lid-driven cavity, 64^3 Q1 hexes (274,625 nodes), elastic sphere R=0.2, N=2 phases, 1 solid"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="fsi", choices=["fsi", "reference"])
    p.add_argument("--precision", default="fp64", choices=["fp32ir", "fp64"],
                   help="the headline arm's arithmetic; the other one runs as a second arm from the same state")
    p.add_argument("--no-other", action="store_true", help="skip the second-precision arm")
    p.add_argument("--no-operators", action="store_true", help="skip the ship/ice per-apply operator rates")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-learned", action="store_true", help="skip the learned-preconditioner arm")
    p.add_argument("--train-steps", type=int, default=4000)
    p.add_argument("--solve-block", default="ns", choices=["ns", "ac", "b"], help="block of --case solve")
    p.add_argument("--smooth-pairs", type=int, default=360,
                   help="synthetic multi-scale training pairs added to the harvested ones")
    p.add_argument("--restart", type=int, default=30, help="GMRES restart length m (<= 64)")
    p.add_argument("--ir-inner-rtol", type=float, default=1e-3,
                   help="relative tolerance of each inner float32 solve of the refinement")
    p.add_argument("--case", default="step", choices=["step", "solve", "pcnet", "batch", "mixed", "operators", "diagnostics", "tet"],
                   help="solve: only a fixed 40-iteration float32-IR NS GMRES solve at 64^3 (a short, "
                        "repeatable launch sequence for ncu captures); pcnet: learned-preconditioner "
                        "applies and training steps at 64^3 with per-kernel timing (JSON on stdout); "
                        "batch: 64 uneven cavity instances, batched launches against per-instance "
                        "launches (JSON on stdout); mixed: 10 steps of the 64^3 cavity in float64 and "
                        "with float32 operators in float64 refinement, per-field drift (JSON on stdout); "
                        "operators: per-apply GDoF/s of every residual and JVP (float64 and float32) "
                        "on the 64^3 cavity, the falling sphere and ship/ice meshes (JSON on stdout); "
                        "diagnostics: centre of mass and tracking of 10^6 points at 64^3 (JSON on stdout)")
    return p.parse_args()


def run_solve_case(precision: str = "fp32ir", block: str = "ns"):
    """Forty Arnoldi steps of one block of the 64^3 cavity (ns, ac: phase 0, b: the solid),
    float32 operator inside float64 refinement (fp32ir: the NS coefficient product in
    float32) or float64 (NS: the first 8 products from the coefficients, the rest through
    element matrices; AC: element matrices from the third product; B: the split operator):
    the launch sequences the profiles under profiles/ were captured on."""
    import torch
    from paper_2402_10348_gb300 import fsi
    from workloads import cavity64
    wl = cavity64()
    d = wl.desc
    dev = torch.device("cuda", 0)
    mesh = fsi.fsi_create_mesh(d)
    fsi.fsi_set_stream(mesh)
    x, xn, xdn = initial_state(fsi, mesh, wl, torch, dev)
    g = torch.Generator(device=dev).manual_seed(0)
    blk, ncomp = {"ns": (fsi.FSI_BLOCK_NS, 4), "ac": (fsi.FSI_BLOCK_AC(0), 1), "b": (fsi.FSI_BLOCK_B(0), 6)}[block]
    if block == "ac":
        fsi.fsi_set_ac_coeffs(mesh, 0, 0.5, 0.0)
    rhs = torch.randn(ncomp * d.nn, dtype=torch.float64, device=dev, generator=g)
    sol = torch.zeros_like(rhs)
    prec = fsi.FSI_PREC_FP32_IR if precision == "fp32ir" else fsi.FSI_PREC_FP64
    o = fsi.solve_opts(m=64, rtol=1e-30, max_iter=40, precision=prec, ir_max=1, ir_inner_rtol=1e-30)
    o.flags |= fsi.FSI_NO_STALL_STOP
    info = fsi.fsi_gmres(mesh, blk, x, xn, xdn, rhs, sol, o, allow_noconv=True)
    torch.cuda.synchronize()
    print(f"solve case ({block}, {precision}): {info.iterations} iterations")


def pc_flops_per_forward(grids, fan):
    """Tensor-core flops of one network forward: 2 x voxels x 27 x in x out channels
    per convolution, with the 16-wide MMA the kernels issue (the output layer's 4
    channels are padded to 16)."""
    lv = {"enc0": 0, "enc1": 1, "enc2": 2, "bot": 3, "dec2": 2, "dec1": 1, "dec0": 0, "out": 0}
    names = ["enc0a", "enc0b", "enc1a", "enc1b", "enc2a", "enc2b", "bota", "botb", "dec2a", "dec2b", "dec1a",
             "dec1b", "dec0a", "dec0b", "out"]
    tot = 0.0
    for name, (co, ci) in zip(names, fan):
        key = name[:-1] if name != "out" else "out"
        nx, ny, nz = grids[lv[key]]
        tot += 2.0 * nx * ny * nz * 27 * ci * 16
    return tot


def run_pcnet_case(applies: int = 20, train_steps: int = 20):
    """The learned preconditioner at 64^3: network applies (pack, 15 tcgen05 convolutions,
    restrictions/prolongations, unpack) and training steps, timed by the library's
    event profiler; the short launch sequence the convolution profile was captured on."""
    import numpy as np
    import torch
    from paper_2402_10348_gb300 import fsi
    from workloads import cavity64, he_normal_weights
    wl = cavity64()
    d = wl.desc
    dev = torch.device("cuda", 0)
    mesh = fsi.fsi_create_mesh(d)
    stream = torch.cuda.current_stream()
    fsi.fsi_set_stream(mesh, stream)
    x, xn, xdn = initial_state(fsi, mesh, wl, torch, dev)
    pc = fsi.fsi_pc_create(mesh, n_pairs_cap=2, linear=True, modulate=True)
    fsi.fsi_pc_set_weights(pc, he_normal_weights(pc.fan, 3))
    g = torch.Generator(device=dev).manual_seed(0)
    r = torch.randn(4 * d.nn, dtype=torch.float64, device=dev, generator=g)
    z = torch.zeros_like(r)
    for _ in range(3):
        fsi.fsi_pc_apply(pc, x, xn, xdn, r, z)
    fsi.fsi_profile(mesh, True)
    for _ in range(applies):
        fsi.fsi_pc_apply(pc, x, xn, xdn, r, z)
    prof_apply = fsi.fsi_profile_read(mesh)
    fsi.fsi_profile(mesh, False)
    # training steps on one stored pair (a product of the operator)
    e = torch.randn(4 * d.nn, dtype=torch.float64, device=dev, generator=g)
    fsi.fsi_jvp(mesh, fsi.FSI_BLOCK_NS, x, xn, xdn, e, r)
    fsi.fsi_pc_add_pair(pc, x, xn, xdn, r, e)
    fsi.fsi_pc_fit_norm(pc)
    fsi.fsi_pc_train(pc, np.zeros(3, dtype=np.int32), 1e-4)
    fsi.fsi_profile(mesh, True)
    fsi.fsi_pc_train(pc, np.zeros(train_steps, dtype=np.int32), 1e-4)
    prof_train = fsi.fsi_profile_read(mesh)
    fsi.fsi_profile(mesh, False)
    pk = peaks()
    fl = pc_flops_per_forward(pc.grids, pc.fan)
    conv = prof_apply["pc_conv"]
    tflops = fl * applies / (conv[1] / 1e3) / 1e12
    out = {"case": "pcnet", "workload": WORKLOAD, "grids": pc.grids, "applies": applies,
           "ms_per_apply": {k: round(v[1] / applies, 4) for k, v in prof_apply.items() if v[0] > 0},
           "conv_launches_per_apply": conv[0] / applies,
           "conv_tflops": round(tflops, 2), "bf16_peak_tflops": pk.get("bf16_tflops"),
           "conv_tensor_frac": round(tflops / pk["bf16_tflops"], 4) if pk.get("bf16_tflops") else None,
           "train_steps": train_steps,
           "ms_per_train_step": {k: round(v[1] / train_steps, 4) for k, v in prof_train.items() if v[0] > 0}}
    print(json.dumps(out), flush=True)


def run_batch_case(count: int = 64, reps: int = 5, steps: int = 3):
    """64 independent cavities of uneven size (16^3 .. 48^3): the float32 NS operator
    applied to all of them in one persistent launch against one launch per instance,
    and the NS solve (Jacobi GMRES(64), float32 operator in float64 refinement, rel-res
    1e-8) batched with a captured restart cycle against one fsi_gmres per instance; then
    `steps` partitioned time steps of all instances, batched against per instance."""
    import torch
    from paper_2402_10348_gb300 import fsi
    from workloads import cavity_batch
    dev = torch.device("cuda", 0)
    wls = cavity_batch(count)
    stream = torch.cuda.Stream()
    meshes, states, rhs = [], [], []
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for wl in wls:
            m = fsi.fsi_create_mesh(wl.desc)
            fsi.fsi_set_stream(m, stream)
            st = initial_state(fsi, m, wl, torch, dev)
            r = torch.zeros(4 * wl.desc.nn, dtype=torch.float64, device=dev)
            fsi.fsi_residual(m, fsi.FSI_BLOCK_NS, *st, r)
            meshes.append(m)
            states.append(st)
            rhs.append(-r)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    b = fsi.fsi_batch_create(meshes, block=fsi.FSI_BLOCK_NS, m=64)
    nodes = sum(wl.desc.nn for wl in wls)
    dof = 4 * nodes
    flags = fsi.FSI_ELASTIC_AUG | fsi.FSI_FP32
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        tm, gm, tuned_us = fsi.fsi_batch_autotune(b, states, flags)
        torch.cuda.synchronize()
        tune_s = time.perf_counter() - t0
    g = torch.Generator(device=dev).manual_seed(0)
    dx = torch.randn(dof, dtype=torch.float64, device=dev, generator=g)
    y = torch.zeros_like(dx)
    parts = [dx[b.offsets[i]:b.offsets[i + 1]] for i in range(count)]
    outs = [y[b.offsets[i]:b.offsets[i + 1]] for i in range(count)]

    def timed(fn, n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            fn()
            e0.record(stream)
            for _ in range(n):
                fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    def per_instance_jvp():
        for i, m in enumerate(meshes):
            fsi.fsi_jvp(m, fsi.FSI_BLOCK_NS, *states[i], parts[i], outs[i], flags)

    ms_single = timed(per_instance_jvp, reps)
    ms_batch = timed(lambda: fsi.fsi_batch_jvp(b, states, dx, y, flags), reps)
    # the solves
    # GMRES(64): these first solves from rest need long restarts (GMRES(30) measured 1.99 s
    # batched and 3.70 s per instance, against 1.42 s and 2.95 s)
    opts = fsi.solve_opts(m=64, rtol=1e-8, max_iter=3000, precision=fsi.FSI_PREC_FP32_IR, ir_inner_rtol=1e-3,
                          ir_max=30)
    rhs_all = torch.cat(rhs).contiguous()
    xb = torch.zeros_like(rhs_all)
    sols = [torch.zeros_like(r) for r in rhs]

    def per_instance_solve():
        its = []
        for i, m in enumerate(meshes):
            its.append(fsi.fsi_gmres(m, fsi.FSI_BLOCK_NS, *states[i], rhs[i], sols[i], opts,
                                     allow_noconv=True).iterations)
        return its

    def batched_solve():
        return [i.iterations for i in fsi.fsi_batch_gmres(b, states, rhs_all, xb, opts, allow_noconv=True)]

    res = {}
    prod_cls = ("ns_jvp_f32", "ns_jvp_f64", "node_sums")
    for name, fn in (("per_instance", per_instance_solve), ("batched_graph", batched_solve)):
        with torch.cuda.stream(stream):
            fn()  # warm-up: workspaces, graph capture
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            its = fn()
            torch.cuda.synchronize()
        res[name] = {"s": round(time.perf_counter() - t0, 4), "iterations_total": int(sum(its)),
                     "iterations_max": int(max(its))}
        # the same solve once more under the library profiler (the batch without its graph:
        # a captured cycle carries no event records): device time and launches of its NS
        # products (element and node kernels), summed over the instances' meshes
        for m in meshes:
            fsi.fsi_profile(m, True)
        fsi.fsi_batch_set_graph(b, False)
        with torch.cuda.stream(stream):
            fn()
        torch.cuda.synchronize()
        fsi.fsi_batch_set_graph(b, True)
        launches, ms = 0, 0.0
        for m in meshes:
            prof = fsi.fsi_profile_read(m)
            fsi.fsi_profile(m, False)
            for c in prod_cls:
                launches += prof.get(c, (0, 0.0))[0]
                ms += prof.get(c, (0, 0.0))[1]
        res[name]["ns_products"] = {"launches": int(launches), "device_ms": round(ms, 3)}
    fsi.fsi_batch_set_graph(b, False)
    with torch.cuda.stream(stream):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its = batched_solve()
        torch.cuda.synchronize()
    res["batched_no_graph"] = {"s": round(time.perf_counter() - t0, 4), "iterations_total": int(sum(its))}
    diff = max(float(torch.linalg.norm(xb[b.offsets[i]:b.offsets[i + 1]] - sols[i]) /
                     max(float(torch.linalg.norm(sols[i])), 1e-300)) for i in range(count))
    out = {"case": "batch", "instances": count, "nodes": nodes, "dof_ns": dof,
           "sizes": sorted(int(wl.desc.nx) for wl in wls), "setup_s": round(setup_s, 2),
           "autotune": {"target_mult": tm, "grid_mult": gm, "best_us": round(tuned_us, 1), "s": round(tune_s, 3)},
           "ns_jvp_f32_public_call": {"per_instance_ms": round(ms_single, 4), "batched_ms": round(ms_batch, 4),
                          "note": "fsi_jvp per instance against fsi_batch_jvp, each call staging its states and "
                                  "building the products' coefficients",
                          "per_instance_gdofs": round(dof / ms_single / 1e6, 3),
                          "batched_gdofs": round(dof / ms_batch / 1e6, 3), "speedup": round(ms_single / ms_batch, 3),
                          "launches_per_instance_arm": 2 * count, "launches_batched": 3},
           "ns_solve_fp32ir_rtol1e-8": res, "max_solution_difference": diff}
    out["time_steps"] = batch_steps(fsi, torch, dev, wls, meshes, stream, steps)
    out["time_steps_learned"] = batch_learned_steps(fsi, torch, dev, wls, meshes, stream, steps=2)
    print(json.dumps(out), flush=True)


def batch_learned_steps(fsi, torch, dev, wls, meshes, stream, steps=2):
    """Batched time steps with flexible GMRES in the NS solves (network and Jacobi directions
    alternately; each instance's network step in one captured graph of parallel branches)
    against batched Jacobi GMRES, from the same initial states (float32 refinement, rel-res
    1e-8).  One network is trained on the largest instance (one harvesting Jacobi step, 360
    synthetic pairs, 4,000 Adam steps; timed apart) and its weights and output scales are
    given to every instance, each keeping its own input scale (from one pair at its state)."""
    import numpy as np
    from workloads import he_normal_weights
    opts = fsi.solve_opts(m=30, rtol=1e-8, max_iter=6000, precision=fsi.FSI_PREC_FP32_IR, ir_inner_rtol=1e-3,
                          ir_max=30)
    big = max(range(len(wls)), key=lambda i: wls[i].desc.nn)
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        st = list(initial_state(fsi, meshes[big], wls[big], torch, dev))
        pct = fsi.fsi_pc_create(meshes[big], n_pairs_cap=512, linear=True, modulate=True)
        fsi.fsi_pc_set_weights(pct, he_normal_weights(pct.fan, 3))
        fsi.fsi_set_pc(meshes[big], pct)
        hv = fsi.solve_opts(m=30, rtol=1e-8, max_iter=6000)
        hv.flags |= fsi.FSI_HARVEST
        fsi.fsi_step(meshes[big], *st, k_max=5, nl_tol=5e-4, solve=hv)
        fsi.fsi_pc_add_smooth_pairs(pct, *st, 360, seed=1)
        fsi.fsi_pc_fit_norm(pct)
        npairs = fsi.fsi_pc_pairs(pct)
        losses = fsi.fsi_pc_train(pct, np.random.default_rng(0).integers(0, npairs, size=4000), 2e-4)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    w = fsi.fsi_pc_get_weights(pct)
    _, kc = fsi.fsi_pc_get_norm(pct)
    pcs = []
    for i, m in enumerate(meshes):
        if i == big:
            pcs.append(pct)
            continue
        with torch.cuda.stream(stream):
            sti = list(initial_state(fsi, m, wls[i], torch, dev))
            pc = fsi.fsi_pc_create(m, n_pairs_cap=1, linear=True, modulate=True)
            fsi.fsi_pc_add_smooth_pairs(pc, *sti, 1, seed=2)  # this instance's input scale
            db, _ = fsi.fsi_pc_get_norm(pc)
            fsi.fsi_pc_set_norm(pc, db, kc)
            fsi.fsi_pc_set_weights(pc, w)
            fsi.fsi_set_pc(m, pc)
        pcs.append(pc)
    torch.cuda.synchronize()
    arms = {}
    for arm in ("jacobi", "learned"):
        with torch.cuda.stream(stream):
            sts = [list(initial_state(fsi, m, wl, torch, dev)) for m, wl in zip(meshes, wls)]
        torch.cuda.synchronize()
        stepper = fsi.fsi_batch_stepper_create(meshes, m=30)
        o = fsi.fsi_solve_opts.from_buffer_copy(opts)
        if arm == "learned":
            o.precond = fsi.FSI_PC_LEARNED
            o.flags |= fsi.FSI_PC_ALTERNATE
        its, stalled, worst = [], 0, 0.0
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for _ in range(steps):
                infos = fsi.fsi_batch_step(stepper, sts, k_max=5, nl_tol=5e-4, solve=o)
                its.append(int(sum(i.gmres_iters_ns for i in infos)))
                stalled += sum(i.stalled_solves for i in infos)
                worst = max(worst, max(i.worst_rel_res for i in infos))
            torch.cuda.synchronize()
        arms[arm] = {"s_per_step_all_instances": round((time.perf_counter() - t0) / steps, 4),
                     "ns_iterations_all_instances": its, "stalled_solves": stalled, "worst_rel_res": worst}
        del stepper
    for m in meshes:
        fsi.fsi_set_pc(m, None)
    return {"trained_on": wls[big].name, "train_s": round(train_s, 2),
            "relative_loss_first_last": [round(float(losses[:50].mean()), 4), round(float(losses[-200:].mean()), 4)],
            "steps": steps, **arms,
            "speedup": round(arms["jacobi"]["s_per_step_all_instances"] / arms["learned"]["s_per_step_all_instances"], 3)}


def batch_steps(fsi, torch, dev, wls, meshes, stream, steps):
    """Partitioned time steps of every instance (float32 operators in float64 refinement,
    Jacobi GMRES(30) to rel-res 1e-8 in every block): one fsi_batch_step per step
    (a batched solve per block kind and nonlinear iteration) against one fsi_step per
    instance and step, from the same initial states."""
    opts = fsi.solve_opts(m=30, rtol=1e-8, max_iter=6000, precision=fsi.FSI_PREC_FP32_IR, ir_inner_rtol=1e-3,
                          ir_max=30)
    arms = {}
    finals = {}
    for arm in ("per_instance", "batched"):
        with torch.cuda.stream(stream):
            sts = [list(initial_state(fsi, m, wl, torch, dev)) for m, wl in zip(meshes, wls)]
        torch.cuda.synchronize()
        stepper = fsi.fsi_batch_stepper_create(meshes, m=30) if arm == "batched" else None
        t0 = time.perf_counter()
        nl, worst, stalled = [], 0.0, 0
        with torch.cuda.stream(stream):
            for _ in range(steps):
                if stepper is not None:
                    infos = fsi.fsi_batch_step(stepper, sts, k_max=5, nl_tol=5e-4, solve=opts)
                else:
                    infos = [fsi.fsi_step(m, *st, k_max=5, nl_tol=5e-4, solve=opts) for m, st in zip(meshes, sts)]
                nl.append(max(i.nl_iters for i in infos))
                worst = max(worst, max(i.worst_rel_res for i in infos))
                stalled += sum(i.stalled_solves for i in infos)
            torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        arms[arm] = {"s_per_step_all_instances": round(dt / steps, 4), "max_nl_iters": nl,
                     "worst_rel_res": worst, "stalled_solves": stalled}
        finals[arm] = [st[1] for st in sts]
        del stepper
    diff = max(float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
               for a, b in zip(finals["batched"], finals["per_instance"]))
    arms["steps"] = steps
    arms["speedup"] = round(arms["per_instance"]["s_per_step_all_instances"] /
                            arms["batched"]["s_per_step_all_instances"], 3)
    arms["max_state_difference"] = diff
    return arms


def operator_rates_of(wl, fsi, torch, dev, reps: int = 3) -> dict:
    """Per-apply GDoF/s of every element operator (residual, float64 and float32 product
    of each block) on one workload's mesh, from a state drawn on the device (phase
    fractions a partition of unity, B near I).  Times come from the library's CUDA-event
    profiler; the NS products stream quadrature-point coefficients built once per state
    (their builds, `op_builds`, are reported apart)."""
    import collections
    d = wl.desc
    nn, N, ns = d.nn, d.n_phase, d.n_solid
    g = torch.Generator(device=dev).manual_seed(0)

    def rnd(*shape):
        return torch.rand(*shape, dtype=torch.float64, device=dev, generator=g)

    x = torch.empty(d.ncomp, nn, dtype=torch.float64, device=dev)
    x[0:3] = 0.2 * (rnd(3, nn) - 0.5)
    x[3] = rnd(nn)
    a = rnd(N, nn) + 0.05
    x[4:4 + N] = 2.0 * a / a.sum(0) - 1.0
    for s in range(ns):
        b0 = 4 + N + 6 * s
        x[b0:b0 + 3] = 1.0 + 0.05 * (rnd(3, nn) - 0.5)
        x[b0 + 3:b0 + 6] = 0.05 * (rnd(3, nn) - 0.5)
    x = x.reshape(-1).contiguous()
    xn = (x + 0.01 * (rnd(x.numel()) - 0.5)).contiguous()
    xdn = (0.1 * (rnd(x.numel()) - 0.5)).contiguous()
    del a
    mesh = fsi.fsi_create_mesh(d)
    fsi.fsi_set_stream(mesh)
    for i in range(N):
        fsi.fsi_set_ac_coeffs(mesh, i, 0.5, 0.1)
    blocks = [("ns", fsi.FSI_BLOCK_NS, 4 * nn)] + [("ac", fsi.FSI_BLOCK_AC(i), nn) for i in range(N)] + \
             [("b", fsi.FSI_BLOCK_B(s), 6 * nn) for s in range(ns)]
    applies, dofs = collections.Counter(), {}
    for profiled in (False, True):  # one untimed pass, then the profiled ones
        if profiled:
            fsi.fsi_profile(mesh, True)
        for kind, blk, n in blocks:
            r = torch.empty(n, dtype=torch.float64, device=dev)
            y = torch.empty(n, dtype=torch.float64, device=dev)
            dx = (rnd(n) - 0.5).contiguous()
            fsi.fsi_residual(mesh, blk, x, xn, xdn, r)
            for _ in range(reps if profiled else 1):
                fsi.fsi_jvp(mesh, blk, x, xn, xdn, dx, y)
            fsi.fsi_residual(mesh, blk, x, xn, xdn, r)
            for _ in range(reps if profiled else 1):
                fsi.fsi_jvp(mesh, blk, x, xn, xdn, dx, y, fsi.FSI_ELASTIC_AUG | fsi.FSI_FP32)
            if profiled:
                applies[f"{kind}_residual"] += 2
                dofs[f"{kind}_residual"] = n
                for cls in (f"{kind}_jvp_f64", f"{kind}_jvp_f32"):
                    applies[cls] += reps
                    dofs[cls] = n
    prof = fsi.fsi_profile_read(mesh)
    fsi.fsi_profile(mesh, False)
    torch.cuda.synchronize()
    ops = {}
    for cls, k in applies.items():
        launches, ms = prof[cls][0], prof[cls][1]
        if ms > 0:
            ops[cls] = {"gdofs": round(dofs[cls] * k / (ms / 1e3) / 1e9, 3),
                        "us_per_apply": round(ms / k * 1e3, 2), "launches_per_apply": launches / k}
    if prof.get("op_builds", (0, 0))[0] > 0:
        ops["op_builds"] = {"us_per_build": round(prof["op_builds"][1] / prof["op_builds"][0] * 1e3, 2),
                            "launches": prof["op_builds"][0]}
    del mesh, x, xn, xdn
    torch.cuda.empty_cache()
    return {"workload": wl.name, "nodes": nn, "phases": N, "solids": ns, "dof_per_node": d.ncomp,
            "unit": "GDoF/s per apply", "ops": ops}


def run_operators_case(reps: int = 3):
    """Per-apply GDoF/s of every element operator at the three single-mesh sizes: the
    64^3 cavity, the falling sphere (96x96x192, 3 phases, 2 solids) and ship/ice
    (256x128x64, 11 phases, 9 solids)."""
    import torch
    from paper_2402_10348_gb300 import fsi
    from workloads import cavity64, falling, shipice
    dev = torch.device("cuda", 0)
    out = {wl.name: operator_rates_of(wl, fsi, torch, dev, reps) for wl in (cavity64(), falling(), shipice())}
    print(json.dumps({"case": "operators", "reps": reps, "unit": "GDoF/s per apply", "configs": out}), flush=True)


def run_tet_case(reps: int = 5):
    """Per-apply device times of the float64 operators on linear tetrahedra (six per box
    cell, interior nodes jittered by 0.2 h): the 64^3 cavity's box (1.57 M elements) and
    the falling sphere's 96x96x192 box (10.6 M elements), on seeded random states.  Each
    apply is an element kernel plus a node-sum kernel; time per apply = class time / calls.
    Inside a 40-iteration NS GMRES the products after the eighth run through the element
    matrices (`ns_jvp_f64_element_matrix`, with the one build's time)."""
    import torch
    from paper_2402_10348_gb300 import fsi
    from workloads import cavity64, falling, random_state, tet_box_mesh
    dev = torch.device("cuda", 0)
    out = {}
    for wl in (cavity64(), falling()):
        d = wl.desc
        X, conn = tet_box_mesh(d, 0.2, seed=1)
        mesh = fsi.fsi_create_tet_mesh(d, X, conn)
        fsi.fsi_set_stream(mesh)
        st = [torch.from_numpy(a.ravel()).to(dev) for a in random_state(d, 0)]
        nn = d.nn
        for i in range(d.n_phase):
            fsi.fsi_set_ac_coeffs(mesh, i, 0.5, 0.1)
        calls = {
            "ns_residual": (lambda y: fsi.fsi_residual(mesh, fsi.FSI_BLOCK_NS, *st, y), 4),
            "ns_jvp_f64": (lambda y: fsi.fsi_jvp(mesh, fsi.FSI_BLOCK_NS, *st, dxs[4], y, fsi.FSI_ELASTIC_AUG), 4),
            "ns_diag": (lambda y: fsi.fsi_diag(mesh, fsi.FSI_BLOCK_NS, *st, y, fsi.FSI_ELASTIC_AUG), 4),
            "ac_jvp_f64": (lambda y: fsi.fsi_jvp(mesh, fsi.FSI_BLOCK_AC(0), *st, dxs[1], y), 1),
            "b_jvp_f64": (lambda y: fsi.fsi_jvp(mesh, fsi.FSI_BLOCK_B(0), *st, dxs[6], y), 6),
        }
        g = torch.Generator(device=dev).manual_seed(0)
        dxs = {c: torch.randn(c * nn, dtype=torch.float64, device=dev, generator=g) for c in (1, 4, 6)}
        res = {}
        for name, (fn, c) in calls.items():
            y = torch.zeros(c * nn, dtype=torch.float64, device=dev)
            fn(y)  # warm
            torch.cuda.synchronize()
            fsi.fsi_profile(mesh, True)
            for _ in range(reps):
                fn(y)
            torch.cuda.synchronize()
            prof = fsi.fsi_profile_read(mesh)
            fsi.fsi_profile(mesh, False)
            ms = prof.get(name, (0, 0.0))[1] / reps
            res[name] = {"ms_per_apply": round(ms, 3), "gdofs": round(c * nn / (ms / 1e3) / 1e9, 3) if ms > 0 else None}
        fsi.fsi_profile(mesh, True)
        for _ in range(reps):
            fsi.fsi_update_ac_coeffs(mesh, 0, *st)
        prof = fsi.fsi_profile_read(mesh)
        fsi.fsi_profile(mesh, False)
        res["gamma_beta"] = {"ms_per_call": round(prof.get("gamma_beta", (0, 0.0))[1] / reps, 3)}
        # inside a solve: after 8 products the NS product runs through element matrices
        rhs = torch.randn(4 * nn, dtype=torch.float64, device=dev, generator=g)
        sol = torch.zeros_like(rhs)
        o = fsi.solve_opts(m=30, rtol=1e-30, max_iter=40)
        o.flags |= fsi.FSI_NO_STALL_STOP
        fsi.fsi_profile(mesh, True)
        fsi.fsi_gmres(mesh, fsi.FSI_BLOCK_NS, *st, rhs, sol, o, allow_noconv=True)
        torch.cuda.synchronize()
        prof = fsi.fsi_profile_read(mesh)
        fsi.fsi_profile(mesh, False)
        em, nd, bld = (prof.get(k, (0, 0.0)) for k in ("ns_jvp_f64_em", "node_sums", "op_builds"))
        if em[0] > 0:
            per = (em[1] + nd[1]) / em[0]
            res["ns_jvp_f64_element_matrix"] = {"ms_per_apply": round(per, 3), "gdofs": round(4 * nn / (per / 1e3) / 1e9, 3),
                                                "applies": em[0], "build_ms": round(bld[1], 3)}
        out[wl.name] = {"elements": int(conn.shape[0]), "nodes": nn, "operators": res}
        if wl.name == "cavity64":
            out[wl.name]["time_steps"] = tet_cavity_steps(fsi, torch, dev, wl, X, conn)
        del mesh
        torch.cuda.empty_cache()
    print(json.dumps({"case": "tet", "reps": reps, "precision": "float64", "configs": out}), flush=True)


def tet_cavity_steps(fsi, torch, dev, wl, X, conn, steps: int = 2):
    """Float64 partitioned time steps of the 64^3 cavity on the tetrahedra of its box
    (jittered nodes), Jacobi GMRES(30) to rel-res 1e-8 in every block.  The initial phase
    indicators come from the grid-cell initialisation on the hexahedral mesh of the same
    box (the tetrahedral mesh has the same nodes, moved by at most 0.2 h)."""
    d = wl.desc
    hexm = fsi.fsi_create_mesh(d)
    fsi.fsi_set_stream(hexm)
    x, xn, xdn = initial_state(fsi, hexm, wl, torch, dev)
    del hexm
    mesh = fsi.fsi_create_tet_mesh(d, X, conn)
    fsi.fsi_set_stream(mesh)
    opts = fsi.solve_opts(m=30, rtol=1e-8, max_iter=6000)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    infos = [fsi.fsi_step(mesh, x, xn, xdn, k_max=wl.k_max, nl_tol=5e-4, solve=opts) for _ in range(steps)]
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"steps": steps, "s_per_step": round(dt / steps, 4), "step_stats": step_stats(infos),
            "finite": bool(torch.isfinite(xn).all())}


def run_diagnostics_case(reps: int = 20):
    """Centre of mass of the solid (Section 5.2) and tracking of 10^6 points (Appendix C)
    on the 64^3 cavity's initial state, CUDA-event times averaged over `reps` calls.
    Algorithmic bytes: the indicator plane (8 B per node) for the centre of mass; per
    point 48 B (read and write of its coordinates) for the tracking, whose gathers of
    8 corners x 3 velocity values hit the L2-resident velocity planes (6.6 MB)."""
    import torch
    from paper_2402_10348_gb300 import fsi
    from workloads import cavity64
    wl = cavity64()
    d = wl.desc
    dev = torch.device("cuda", 0)
    mesh = fsi.fsi_create_mesh(d)
    stream = torch.cuda.current_stream()
    fsi.fsi_set_stream(mesh, stream)
    x, _, _ = initial_state(fsi, mesh, wl, torch, dev)
    x[0:3 * d.nn] = 0.1 * torch.rand(3 * d.nn, dtype=torch.float64, device=dev)
    npts = 1_000_000
    g = torch.Generator(device=dev).manual_seed(0)
    pts = torch.rand(npts, 3, dtype=torch.float64, device=dev, generator=g)
    com = fsi.fsi_center_of_mass(mesh, x, 0)
    fsi.fsi_track_points(mesh, x, pts)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fsi.fsi_center_of_mass(mesh, x, 0)  # synchronises (host reads the result)
    e1.record(stream)
    torch.cuda.synchronize()
    com_us = e0.elapsed_time(e1) / reps * 1e3
    e0.record(stream)
    for _ in range(reps):
        fsi.fsi_track_points(mesh, x, pts)
    e1.record(stream)
    torch.cuda.synchronize()
    trk_us = e0.elapsed_time(e1) / reps * 1e3
    trk_bytes = npts * 48
    print(json.dumps({"case": "diagnostics", "workload": WORKLOAD, "center_of_mass": [round(c, 6) for c in com],
                      "center_of_mass_us": round(com_us, 2), "center_of_mass_bytes": 8 * d.nn,
                      "points": npts, "track_us": round(trk_us, 2),
                      "track_gbs": round(trk_bytes / (trk_us * 1e-6) / 1e9, 1),
                      "note": "center_of_mass includes its device-to-host copy and synchronisation"}), flush=True)


def run_mixed_case(steps: int = 100):
    """The 64^3 cavity from its initial state: `steps` time steps with float64 operators
    and, from the same state, with float32 operators inside float64 refinement (both
    Jacobi GMRES(30) to rel-res 1e-8); the relative L2 distance of v, p, phi and B after
    every step, and the time per step of each."""
    import torch
    from paper_2402_10348_gb300 import fsi
    from workloads import cavity64
    wl = cavity64()
    d = wl.desc
    dev = torch.device("cuda", 0)
    out = {"case": "mixed", "workload": WORKLOAD, "steps": steps}
    states = {}
    for name, prec in (("fp64", fsi.FSI_PREC_FP64), ("fp32ir", fsi.FSI_PREC_FP32_IR)):
        mesh = fsi.fsi_create_mesh(d)
        fsi.fsi_set_stream(mesh)
        x, xn, xdn = initial_state(fsi, mesh, wl, torch, dev)
        solve = fsi.solve_opts(m=30, rtol=1e-8, max_iter=6000, precision=prec, ir_inner_rtol=1e-3, ir_max=30)
        hist = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            fsi.fsi_step(mesh, x, xn, xdn, k_max=wl.k_max, nl_tol=5e-4, solve=solve)
            hist.append(xn.clone())
        torch.cuda.synchronize()
        out[name + "_s_per_step"] = round((time.perf_counter() - t0) / steps, 4)
        states[name] = hist
    nn = d.nn
    fields = {"v": (0, 3), "p": (3, 4), "phi": (4, 4 + d.n_phase), "B": (4 + d.n_phase, d.ncomp)}
    drift = {k: [] for k in fields}
    for a, b in zip(states["fp64"], states["fp32ir"]):
        for k, (c0, c1) in fields.items():
            ref = a[c0 * nn:c1 * nn]
            drift[k].append(float(torch.linalg.norm(b[c0 * nn:c1 * nn] - ref) / torch.linalg.norm(ref)))
    out["relative_l2_fp32ir_vs_fp64_per_step"] = {k: [float(f"{v:.2e}") for v in vs] for k, vs in drift.items()}
    out["max_over_steps"] = {k: float(f"{max(vs):.2e}") for k, vs in drift.items()}
    print(json.dumps(out), flush=True)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(value: float, world: int, device=None) -> float:
    """Max over ranks (identity at world size 1)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float, world: int, device=None) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
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
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        out.update(sm_mhz=float(np.median(sm)) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=reasons, samples=len(rows))
        return out


# ---------------------------------------------------------------- roofline data
# Algorithmic float operations per element of one element evaluation (no halo
# recomputation), counted from the arithmetic of the kernels' element functions;
# multiply by the elements of one launch.
def flops_per_element(kernel: str, n_solid: int) -> float:
    """The float64 NS product through element matrices: 2 x 32 x 32 per element.  Per
    quadrature point: the NS product from frozen coefficients 486 + 114 with solids
    (interpolation of dv, dp: 172; convective and mass terms 54; stresses 92; the
    elastic linearization 114; test-function scatter 166), its coefficient build
    635 + 167 per solid, NS residual 635 + 167 per solid, AC JVP 247, B JVP 892; 8
    points per element."""
    if kernel == "ns_jvp_f64_em":
        return 2.0 * 32 * 32  # the element matrix applied: 1024 FMAs per element
    per_qp = {"ns_jvp": 486 + (114 if n_solid > 0 else 0), "op_builds": 0,
              "ns_residual": 635 + 167 * n_solid, "ac_jvp": 247, "b_jvp": 892}
    for k, v in per_qp.items():
        if kernel.startswith(k):
            return 8.0 * v
    return 0.0


def operator_rates(prof: dict, nn: int) -> dict:
    """GDoF/s of each element-operator class over the profiled steps: block DoF per
    launch (NS 4 nn, one AC phase nn, one solid's B 6 nn) x launches / summed event
    time.  One launch is one apply on a mesh whose solids fit one operator pass (the
    cavity's one solid does)."""
    dof = {"ns": 4 * nn, "ac": nn, "b": 6 * nn}
    out = {}
    for k, (launches, ms) in prof.items():
        kind = k.split("_")[0]
        if kind not in dof or not ("_jvp_" in k or k.endswith("_residual")) or launches <= 0 or ms <= 0:
            continue
        out[k] = {"gdofs": round(dof[kind] * launches / (ms / 1e3) / 1e9, 3),
                  "us_per_launch": round(ms / launches * 1e3, 2)}
    return out


def peaks(measured=None):
    """Roofline denominators: HBM from MEASURED_PEAKS.json (a measured copy figure),
    float32 / float64 FMA rates from fsi_probe_peaks on this GPU in the same run (else
    derived from unit counts: 152 SMs x 128 FP32 lanes, 2 DFMA per clock, x 2 flop x
    the maximum SM clock)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    pk = {}
    if os.path.exists(path):
        pk = json.load(open(path))
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    out = {
        "hbm_gbs": pk.get("hbm_gbs", 6800.0),
        "hbm_src": "measured" if "hbm_gbs" in pk else "fallback",
        "fp32_tflops": 152 * 128 * 2 * sm_mhz * 1e6 / 1e12,
        "fp64_tflops": 152 * 2 * 2 * sm_mhz * 1e6 / 1e12,
        "alu_src": "derived: 152 SMs x FMA lanes per SM x 2 flop x max SM clock",
        "bf16_tflops": pk.get("bf16_tflops", 1900.0),
        "bf16_src": "measured (cuBLAS bf16 burst)" if "bf16_tflops" in pk else "fallback",
    }
    if measured:
        out.update(fp32_tflops=measured["fp32_tflops"], fp64_tflops=measured["fp64_tflops"],
                   alu_src="measured in this run (fsi_probe_peaks: 8 independent FMA chains per thread)")
    return out


def traffic_record(kernel: str):
    """ncu DRAM bytes per launch of a kernel class, from profiles/traffic.json, used
    only while the source file it was measured on is unchanged (sha256 match)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(kernel)
    if not rec:
        return None
    h = hashlib.sha256()
    for s in rec["sources"]:
        src = os.path.join(ROOT, s)
        if not os.path.exists(src):
            return None
        h.update(open(src, "rb").read())
    return rec if h.hexdigest() == rec["sha256"] else None


def roofline(name, launches, ms, nbytes, d, pk, basis_f64=True):
    """Roofline of one kernel class over the timed region.  Vector (Krylov) classes:
    the algorithmic bytes their launch sites declare against the HBM peak.  Element
    operators: the flop count of one element evaluation times the elements of a launch
    against the FMA peak of their precision and, where the launch declares its bytes
    (the NS product streams its coefficients), those bytes against the HBM peak; the
    roof with the longer minimum time binds and is the one reported."""
    if launches <= 0 or ms <= 0:
        return None
    out = {"kernel": name, "launches": launches, "avg_launch_us": round(ms / launches * 1e3, 2)}
    t = ms / launches / 1e3  # s per launch
    fpe = flops_per_element(name, d.n_solid)
    rec = traffic_record(name)
    hbm = alu = None
    if nbytes > 0:
        b = nbytes / launches
        hbm = {"bound": "hbm", "achieved": round(b / t / 1e9, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
               "frac": round(b / t / 1e9 / pk["hbm_gbs"], 4), "algorithmic_bytes_per_launch": round(b),
               "t_min_us": b / (pk["hbm_gbs"] * 1e9) * 1e6,
               "peak_src": pk["hbm_src"] + " (MEASURED_PEAKS.json copy, read+write)"}
    if fpe > 0:
        flops = fpe * d.ne
        peak = pk["fp32_tflops"] if name.endswith("f32") else pk["fp64_tflops"]
        alu = {"bound": "alu", "achieved": round(flops / t / 1e12, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
               "frac": round(flops / t / 1e12 / peak, 4), "algorithmic_flops_per_launch": flops,
               "t_min_us": flops / (peak * 1e12) * 1e6, "peak_src": pk.get("alu_src", "derived")}
    elif hbm is not None and basis_f64 and (name.startswith("krylov_dot") or name.startswith("krylov_update")):
        # float64 projections and updates do one float64 FMA per float64 element read
        tf = nbytes / launches / 8.0 * 2.0 / t / 1e12
        out["alu_fp64"] = {"achieved": round(tf, 3), "peak": round(pk["fp64_tflops"], 3), "unit": "TFLOP/s",
                           "frac": round(tf / pk["fp64_tflops"], 4), "peak_src": pk.get("alu_src", "derived")}
    bind = max([r for r in (hbm, alu) if r is not None], key=lambda r: r["t_min_us"], default=None)
    if bind is None:
        return out
    other = alu if bind is hbm else hbm
    out.update({k: v for k, v in bind.items() if k != "t_min_us"})
    if other is not None:
        out["other_roof"] = {k: v for k, v in other.items() if k != "t_min_us"}
    traffic = None
    if rec is not None:
        traffic = rec.get("traffic_per_launch")
        if traffic is None and "traffic_ratio" in rec and nbytes > 0:
            traffic = round(rec["traffic_ratio"] * nbytes / launches)
        out["traffic_note"] = rec["note"]
    out["traffic"] = traffic
    return out


# ---------------------------------------------------------------- the GPU arm
def initial_state(fsi, mesh, wl, torch, dev):
    d = wl.desc
    nn, nc = d.nn, d.ncomp
    phi = torch.zeros(d.n_phase * nn, dtype=torch.float64, device=dev)
    fsi.fsi_init_phases(mesh, wl.surfaces, wl.rules, wl.grid_cells, phi)
    x = torch.zeros(nc * nn, dtype=torch.float64, device=dev)
    x[4 * nn:(4 + d.n_phase) * nn] = phi
    base = 4 + d.n_phase
    for s in range(d.n_solid):
        x[(base + 6 * s) * nn:(base + 6 * s + 3) * nn] = 1.0
    return x, x.clone(), torch.zeros_like(x)


FIELDS_OF = lambda d: {"v": (0, 3), "p": (3, 4), "phi": (4, 4 + d.n_phase), "B": (4 + d.n_phase, d.ncomp)}


def field_errors(d, got, ref):
    """Relative L2 distance per field (v, p, phi, B) of two state vectors."""
    import torch
    nn = d.nn
    out = {}
    for k, (c0, c1) in FIELDS_OF(d).items():
        r = ref[c0 * nn:c1 * nn]
        out[k] = float(f"{float(torch.linalg.norm(got[c0 * nn:c1 * nn] - r) / torch.linalg.norm(r)):.3e}")
    return out


def step_stats(infos):
    return {"nl_iters": [i.nl_iters for i in infos],
            "gmres_iters_ns": [i.gmres_iters_ns for i in infos],
            "gmres_iters_ac": [i.gmres_iters_ac for i in infos],
            "gmres_iters_b": [i.gmres_iters_b for i in infos],
            "worst_rel_res": max(i.worst_rel_res for i in infos),
            "stalled_solves": sum(i.stalled_solves for i in infos)}


def run_gpu(args):
    import torch
    from paper_2402_10348_gb300 import fsi
    from workloads import cavity64

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    wl = cavity64()
    d = wl.desc
    measured = fsi.fsi_probe_peaks()  # FMA rates and bandwidths of this GPU, before the run
    mesh = fsi.fsi_create_mesh(d, device=local)
    stream = torch.cuda.current_stream()
    fsi.fsi_set_stream(mesh, stream)
    f64 = args.precision == "fp64"
    prec = fsi.FSI_PREC_FP64 if f64 else fsi.FSI_PREC_FP32_IR

    def opts(p):
        return fsi.solve_opts(m=args.restart, rtol=1e-8, max_iter=6000, precision=p,
                              ir_inner_rtol=args.ir_inner_rtol, ir_max=30)

    solve = opts(prec)
    x, xn, xdn = initial_state(fsi, mesh, wl, torch, dev)

    def step(o=solve):
        return fsi.fsi_step(mesh, x, xn, xdn, k_max=wl.k_max, nl_tol=5e-4, solve=o)

    # the learned preconditioner of the NS block: training pairs are harvested from the
    # (untimed) Jacobi warm-up steps
    pc = None
    if not args.no_learned:
        from workloads import he_normal_weights
        pc = fsi.fsi_pc_create(mesh, n_pairs_cap=512, linear=True, modulate=True)
        fsi.fsi_pc_set_weights(pc, he_normal_weights(pc.fan, 3))
        fsi.fsi_set_pc(mesh, pc)
        harvest = opts(prec)
        harvest.flags |= fsi.FSI_HARVEST
    for _ in range(args.warmup):
        step(harvest if pc is not None else solve)
    torch.cuda.synchronize()
    snapshot = (x.clone(), xn.clone(), xdn.clone())

    def restore():
        for a, b in zip((x, xn, xdn), snapshot):
            a.copy_(b)
        torch.cuda.synchronize()

    clocks = Clocks(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    dof, infos = 0, []
    for _ in range(args.steps):
        inf = step()
        dof += inf.dof_applied
        infos.append(inf)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms_local = e0.elapsed_time(e1)
    final = (x.clone(), xn.clone(), xdn.clone())
    # the same steps again from the same state with every launch bracketed by CUDA
    # events (the library's profiler): per-class launch counts and device times.  The
    # solver is deterministic, so the replay runs the timed region's launches; the
    # events cost host time per launch and are kept out of the timed region itself.
    restore()
    fsi.fsi_profile(mesh, True)
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    replay = [step() for _ in range(args.steps)]
    r1.record(stream)
    torch.cuda.synchronize()
    prof = fsi.fsi_profile_read(mesh)
    fsi.fsi_profile(mesh, False)
    clk = clocks.stop()
    replay_same = all(a.gmres_iters_ns == b.gmres_iters_ns and a.gmres_iters_ac == b.gmres_iters_ac
                      and a.gmres_iters_b == b.gmres_iters_b and a.nl_iters == b.nl_iters
                      for a, b in zip(infos, replay))
    replay_same = replay_same and all(bool(torch.equal(a, b)) for a, b in zip((x, xn, xdn), final))
    profiled = {"ms_per_step": round(r0.elapsed_time(r1) / args.steps, 3), "identical_to_timed": replay_same}
    ms = reduce_max(ms_local, world, dev)
    dof_all = reduce_sum(float(dof), world, dev)
    seconds = ms / 1e3
    value = dof_all / seconds / 1e9
    launches = int(sum(v[0] for v in prof.values()))

    # dominant kernel class (largest summed event time) and its roofline; the
    # dominant operator kernel is reported beside it
    pk = peaks(measured)
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    roof = roofline(dom[0], *dom[1], d, pk, basis_f64=f64)
    ops = {k: v for k, v in prof.items() if flops_per_element(k, d.n_solid) > 0 and v[0] > 0}
    roof_op = None
    if ops:
        oname, ov = max(ops.items(), key=lambda kv: kv[1][1])
        roof_op = roofline(oname, *ov, d, pk, basis_f64=f64)

    # the other precision from the same state: float32 operators inside float64
    # refinement against the float64 headline (or the reverse), same steps
    other = None
    if rank == 0 and not args.no_other:
        oprec = fsi.FSI_PREC_FP32_IR if f64 else fsi.FSI_PREC_FP64
        restore()
        oo = opts(oprec)
        step(oo)  # first use allocates the float32 staging
        restore()
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        oinfos = [step(oo) for _ in range(args.steps)]
        q1.record(stream)
        torch.cuda.synchronize()
        oms = q0.elapsed_time(q1)
        odof = sum(i.dof_applied for i in oinfos)
        other = {"precision": "fp32ir" if f64 else "fp64",
                 "value": round(odof / (oms / 1e3) / 1e9, 5), "unit": UNIT,
                 "s_per_timestep": round(oms / args.steps / 1e3, 5),
                 "step_stats": step_stats(oinfos),
                 ("error_vs_fp64" if f64 else "error_vs_fp32ir"): field_errors(d, xn, final[1])}
        # one profiled step of this precision: its NS product's roofline
        restore()
        fsi.fsi_profile(mesh, True)
        step(oo)
        torch.cuda.synchronize()
        oprof = fsi.fsi_profile_read(mesh)
        fsi.fsi_profile(mesh, False)
        oname = "ns_jvp_f32" if f64 else "ns_jvp_f64_em"
        if oprof.get(oname, (0, 0))[0] > 0:
            other["roofline_ns_product"] = roofline(oname, *oprof[oname], d, pk, basis_f64=not f64)
        other["kernel_ms_one_step"] = {k: [v[0], round(v[1], 3)] for k, v in oprof.items() if v[0] > 0}

    learned = None
    if pc is not None:
        learned = run_learned_arm(fsi, torch, mesh, pc, solve, step, (x, xn, xdn), snapshot, args, stream)
        learned["jacobi_s_per_timestep"] = round(ms / args.steps / 1e3, 5)
        learned["jacobi_ns_iters"] = [i.gmres_iters_ns for i in infos]
        learned["jacobi_nl_iters"] = [i.nl_iters for i in infos]
        learned["jacobi_worst_rel_res"] = max(i.worst_rel_res for i in infos)
        learned["faster_than_jacobi"] = learned["s_per_timestep"] < learned["jacobi_s_per_timestep"]

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(fsi, mesh, wl, torch, dev, stream, step_fn=lambda xs: fsi.fsi_step(
            mesh, *xs, k_max=wl.k_max, nl_tol=5e-4, solve=solve), steps=max(1, min(args.steps, 2)), world=world)
    del mesh, pc
    torch.cuda.empty_cache()
    shipice_ops = None
    if rank == 0 and not args.no_operators:
        from workloads import shipice
        shipice_ops = operator_rates_of(shipice(), fsi, torch, dev, reps=2)

    line = {
        "metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if f64 else "f32",
        "precision": ("float64 throughout (operators, Arnoldi basis, reductions, Hessenberg and Givens)" if f64 else
                      "float32 operator applies and float32 Arnoldi basis inside float64 iterative "
                      "refinement; float64 residuals, reductions, Hessenberg and Givens"),
        "data": "synthetic (seeded icosphere surface, initial phases by the grid-cell method)",
        "config": {"workload": WORKLOAD, "nodes": d.nn, "dof_per_node": d.ncomp, "dt": d.dt,
                   "nl_iters_max": wl.k_max,
                   "gmres": f"Jacobi GMRES({args.restart}) rtol 1e-8 (NS block of the enclosed cavity: the pin "
                            "node keeps its continuity equation, pressure shifted to p = 0 there after the solve)"
                   + (f"; inner solves to {args.ir_inner_rtol:g}" if not f64 else ""),
                   "l2": ("inputs larger than L2: a time step streams the 64^3 state, the quadrature-point "
                          "coefficients of the NS product "
                          f"({d.ne * 8 * 44 * (8 if f64 else 4) / 1e6:.0f} MB) and the (m+1) x 1.1M Krylov basis "
                          f"({(args.restart + 1) * 4 * d.nn * (8 if f64 else 4) / 1e6:.0f} MB) every restart cycle, "
                          "against a 129 MB L2"),
                   "parallelism": f"replicas x{world}"},
        "s_per_timestep": round(ms / args.steps / 1e3, 5),
        "step_stats": step_stats(infos),
        "gpu_launches": launches,
        "profiled_replay": profiled,
        "kernel_ms": {k: [v[0], round(v[1], 3)] for k, v in prof.items() if v[0] > 0},
        "operator_gdofs": operator_rates({k: (v[0], v[1]) for k, v in prof.items()}, d.nn),
        "roofline": roof,
        "roofline_operator": roof_op,
        "measured_peaks": {k: round(v, 2) for k, v in measured.items()},
        "clocks": clk,
        "e2e": e2e,
        "other_precision": other,
        "learned_pc": learned,
        "shipice_operators": shipice_ops,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_learned_arm(fsi, torch, mesh, pc, solve, step, state, snapshot, args, stream):
    """Trains the network on the harvested pairs plus synthetic multi-scale pairs at the
    warm-up's final state (timed apart), then replays the timed steps from the same
    initial state with flexible GMRES on the NS block whose directions alternate between
    the network and Jacobi (Jacobi on the other blocks, and as the fallback);
    s/timestep to rel-res 1e-8."""
    import numpy as np
    x, xn, xdn = state
    harvested = fsi.fsi_pc_pairs(pc)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if args.smooth_pairs > 0:
        fsi.fsi_pc_add_smooth_pairs(pc, x, xn, xdn, args.smooth_pairs, seed=1)
    npairs = fsi.fsi_pc_pairs(pc)
    fsi.fsi_pc_fit_norm(pc)
    rng = np.random.default_rng(0)
    order = rng.integers(0, npairs, size=args.train_steps)
    losses = fsi.fsi_pc_train(pc, order, 2e-4)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    opts = fsi.fsi_solve_opts.from_buffer_copy(solve)
    opts.precond = fsi.FSI_PC_LEARNED
    opts.flags |= fsi.FSI_PC_ALTERNATE

    def restore():
        for dst, src in zip((x, xn, xdn), snapshot):
            dst.copy_(src)

    restore()
    step(opts)  # first use allocates the flexible-GMRES directions
    restore()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = [step(opts) for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    # the same network inside float32 refinement: flexible inner solves (alternate directions)
    o32 = fsi.fsi_solve_opts.from_buffer_copy(opts)
    o32.precision = fsi.FSI_PREC_FP32_IR
    o32.ir_inner_rtol = args.ir_inner_rtol
    o32.ir_max = 30
    restore()
    step(o32)  # first use of the float32 staging with the network
    restore()
    torch.cuda.synchronize()
    e0.record(stream)
    infos32 = [step(o32) for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    ms32 = e0.elapsed_time(e1)
    fp32ir = {"s_per_timestep": round(ms32 / args.steps / 1e3, 5), "ns_iters": [i.gmres_iters_ns for i in infos32],
              "worst_rel_res": max(i.worst_rel_res for i in infos32),
              "fallback_solves": [i.fallback_solves for i in infos32]}
    return {
        "float32_refinement": fp32ir,
        "network": "U-Net, 4 levels, 16 channels, 3x3x3 convolutions (tcgen05, bf16 x bf16 -> f32), "
                   "linear (no activation), inputs modulated by the solid indicator",
        "directions": "flexible GMRES, network and Jacobi directions alternately",
        "pairs": npairs, "pairs_harvested": harvested, "pairs_smooth": npairs - harvested,
        "train_steps": args.train_steps, "train_s": round(train_s, 3),
        "train_ms_per_step": round(1e3 * train_s / max(1, args.train_steps), 3),
        "relative_loss_first_last": [round(float(losses[:50].mean()), 4), round(float(losses[-200:].mean()), 4)],
        "s_per_timestep": round(ms / args.steps / 1e3, 5),
        "nl_iters": [i.nl_iters for i in infos],
        "ns_iters": [i.gmres_iters_ns for i in infos],
        "max_ratio": [i.max_ratio for i in infos],
        "worst_rel_res": max(i.worst_rel_res for i in infos),
        "stalled_solves": [i.stalled_solves for i in infos],
        "fallback_solves": [i.fallback_solves for i in infos],
    }


def run_e2e(fsi, mesh, wl, torch, dev, stream, step_fn, steps, world):
    """Same metric through the C ABI with the state in pinned HOST memory: every step
    copies x^n, dx^n (and x^{n+1}) to the device, runs the step and copies the new
    state back (the step's result)."""
    d = wl.desc
    n = d.ncomp * d.nn
    host = [torch.empty(n, dtype=torch.float64, pin_memory=True) for _ in range(3)]
    xs = initial_state(fsi, mesh, wl, torch, dev)
    for h, t in zip(host, xs):
        h.copy_(t)
    dev_bufs = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(3)]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    dof = 0
    for _ in range(steps):
        for db, h in zip(dev_bufs, host):
            db.copy_(h, non_blocking=True)
        inf = step_fn(dev_bufs)
        dof += inf.dof_applied
        for db, h in zip(dev_bufs, host):
            h.copy_(db, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = reduce_max(e0.elapsed_time(e1), world, dev)
    dof = reduce_sum(float(dof), world, dev)
    return {"value": round(dof / (ms / 1e3) / 1e9, 5), "unit": UNIT, "steps": steps,
            "h2d_bytes_per_step": 3 * n * 8, "d2h_bytes_per_step": 3 * n * 8}


# ---------------------------------------------------------------- the oracle on the host cores
def _oracle_sample(nz_slab: int, seed: int = 0):
    """A z-slab of the 64^3 cavity (same spacing, physics and a seeded state)."""
    from workloads import cavity64, random_state
    wl = cavity64()
    d = wl.desc
    d.nz = nz_slab
    d.lz = nz_slab * (1.0 / 64.0)
    x1, xn, xdn = random_state(d, seed)
    return d, (x1, xn, xdn)


def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(budget_s: float = 3.0):
    """The oracle on the host cores.  Per-apply rates of its NS, AC and B products on a
    64 x 64 x 16-element slab of the workload (about budget_s each; `value` is the NS
    product's, the dominant apply of a step), and the wall time of one nonlinear
    iteration of the 16^3 cavity's first time step (NS, both AC and the B block solved
    by the oracle's Jacobi GMRES(30) to 1e-8, the NS block without the pin row plus the
    pressure shift)."""
    from oracle import blocks, step
    from oracle.fields import Problem, State
    from oracle.gridcell import apply_rules, signed_distance_phi
    from workloads import cavity16
    d, (x1, xn, xdn) = _oracle_sample(16)
    pb, st = Problem(d), State(x1, xn, xdn)
    rng = np.random.default_rng(1)
    coeffs = {"gamma": {i: 0.5 for i in range(d.n_phase)}, "beta": {i: 0.1 for i in range(d.n_phase)}}
    rates = {}
    for name, blk, ncomp in (("ns", "ns", 4), ("ac", ("ac", 1), 1), ("b", ("b", 0), 6)):
        dx = rng.normal(size=ncomp * d.nn)
        t0 = time.perf_counter()
        reps = 0
        while True:
            blocks.jvp(pb, st, blk, dx, coeffs)
            reps += 1
            if time.perf_counter() - t0 > budget_s:
                break
        dt = time.perf_counter() - t0
        rates[name + "_jvp"] = {"gdofs": round(reps * ncomp * d.nn / dt / 1e9, 7), "applies": reps,
                                "s_per_apply": round(dt / reps, 3)}
    wl = cavity16()
    dd = wl.desc
    phi, _ = signed_distance_phi(dd, wl.surfaces[0], dd.eps, wl.grid_cells)
    x = np.zeros((dd.ncomp, dd.nn))
    x[4:4 + dd.n_phase] = apply_rules(dd, {0: phi}, wl.rules, dd.eps)
    x[4 + dd.n_phase: 4 + dd.n_phase + 3] = 1.0
    s16 = State(x.copy(), x.copy(), np.zeros_like(x))
    t0 = time.perf_counter()
    info = step.time_step(Problem(dd), s16, step.StepOptions(k_max=1, rtol=1e-8, max_iter=3000, pin_shift=True))
    it_s = time.perf_counter() - t0
    return {"value": rates["ns_jvp"]["gdofs"], "unit": UNIT, "cores": os.cpu_count(), "cpu_model": _cpu_model(),
            "kind": "oracle",
            "sample": f"float64 numpy oracle (BLAS may use all {os.cpu_count()} cores): NS, AC and B products on "
                      f"a 64x64x16-element slab of the 64^3 cavity (about {budget_s:.0f} s each; value = NS); one "
                      "nonlinear iteration of the 16^3 cavity's first step",
            "per_apply": rates,
            "cavity16_one_nonlinear_iteration_s": round(it_s, 2),
            "cavity16_gmres_iters": {k: v[0] for k, v in info.gmres_iters.items()}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import ns
    from oracle.fields import Problem, State
    d, (x1, xn, xdn) = _oracle_sample(4)
    pb, st = Problem(d), State(x1, xn, xdn)
    dx = np.random.default_rng(1).normal(size=(4, d.nn))
    for _ in range(args.warmup):
        ns.ns_jvp(pb, st, dx)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ns.ns_jvp(pb, st, dx)
    dt = time.perf_counter() - t0
    value = args.steps * 4 * d.nn / dt / 1e9
    sample = (f"each step: one float64 NS Jacobian-vector product of the oracle on a 64x64x4-element slab "
              f"of the 64^3 cavity ({4 * d.nn} DoF)")
    line = {"metric": METRIC, "value": round(value, 7), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample}, "impl": "reference",
            "cpu_baseline": {"value": round(value, 7), "unit": UNIT, "kind": "oracle", "cores": os.cpu_count(),
                             "sample": sample},
            "e2e": {"value": round(value, 7), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.case == "pcnet":
        run_pcnet_case()
    elif args.case == "batch":
        run_batch_case(steps=args.steps if "--steps" in sys.argv else 3)
    elif args.case == "mixed":
        run_mixed_case(args.steps if "--steps" in sys.argv else 100)
    elif args.case == "operators":
        run_operators_case()
    elif args.case == "diagnostics":
        run_diagnostics_case()
    elif args.case == "tet":
        run_tet_case()
    elif args.case == "solve":
        run_solve_case(args.precision if "--precision" in sys.argv else "fp32ir", args.solve_block)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
