#!/usr/bin/env python3
"""Benchmark of the gradient-enhanced damage hot path on one GB300 per rank.

Metric: qp constitutive+assembly updates/s and Newton-step ms.  One bench step
is one quasi-static load step of the monolithic scheme: Newton iterations, each
an element-kernel pass (kinematics, ICNN energy with derivatives, yield network
and local damage update, degraded stress, residual and consistent tangent,
CSR scatter), the residual norms, a Jacobi-preconditioned BiCGStab solve and a
backtracking line search.  value = (#qp x Newton iterates in the timed steps) /
(timed device time), an iterate being the first pass of a (sub)step or the
accepted pass of a Newton direction: whole-step throughput, inputs resident in
HBM.  Rejected line-search trials are timed but not counted.

Workloads (synthetic, seeded; see paper_2604_03411_gb300/inputs.py):
  notched   2D notched plate 2:1, graded Q4 mesh of 39,936 elements (159,744 qp),
            both ICNNs width 32, 50 steps to 60% nominal strain, FP64 (default)
  cube      3D cube, 64^3 HEX8 (2,097,152 qp), biaxial, both ICNNs width 64
  square    2D 8x8 Q4 square, load-unload-reload
  batch     96 independent Q4 specimens (16..96 x 16..48 elements, widths 16/24/32,
            20..60 steps each) in one batched handle, mixed precision; under
            torchrun the specimens are split across the ranks (strong scaling)

Multi-GPU: one process per GPU under torchrun; a single mesh does not shard, so
every rank runs an independent replica of the workload (weak scaling) and
value sums the ranks' qp updates over the slowest rank's time.  The batch
workload shards its specimens instead (no collective on the data path).

--impl reference times the FP64 CPU oracle (the project's reference
implementation of the method) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "qp constitutive+assembly updates/s & Newton-step ms, mixed vs FP64, 1 GB300"
UNIT = "qp-updates/s"
L2_FLUSH_BYTES = 512 << 20          # > 129 MB L2
FP64_PEAK_TFLOPS_NOMINAL = 1.25     # GB300 dense FP64 (nominal, the recipe's table)
FP32_PEAK_TFLOPS_NOMINAL = 152 * 128 * 2 * 2.07e9 / 1e12   # 80.5: SMs x FP32 lanes x FMA x max clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gd", choices=["gd", "reference"])
    ap.add_argument("--workload", default="notched", choices=["notched", "notched3d", "cube", "square", "batch"])
    ap.add_argument("--precision", default=None, choices=["fp64", "mixed"],
                    help="default: fp64 (mixed for the batch workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true",
                    help="FP64 runs only: skip the mixed-precision comparison on the same steps")
    ap.add_argument("--inner", default="auto", choices=["auto", "fp64", "refined"],
                    help="Newton inner-solve policy (gd_options.inner_solve)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--coarse", type=int, default=None,
                    help="coarse unknowns of the two-level preconditioner (gd_options.coarse; 0 = Jacobi only)")
    return ap.parse_args()


def make_workload(name, rank=0, world=1):
    from paper_2604_03411_gb300 import inputs as I
    if name == "batch":
        from paper_2604_03411_gb300 import shard
        allp = I.config5()
        mine = shard.shard(allp, rank, world)
        ps = [allp[i] for i in mine]
        desc = {"workload": "batch_96_specimens_q4", "specimens": len(allp), "specimens_this_rank": len(ps),
                "elements": sum(p.mesh.n_elems for p in ps), "qp": sum(p.mesh.n_elems * 4 for p in ps),
                "dofs": sum(p.mesh.n_nodes * 3 for p in ps), "icnn_width": "16/24/32 per specimen",
                "load_steps": "20..60 per specimen", "length_scale": 0.1}
        return ps, desc
    if name == "notched":
        p = I.config2()
        desc = {"workload": "notched_plate_q4", "elements": p.mesh.n_elems, "qp": p.mesh.n_elems * 4,
                "dofs": p.mesh.n_nodes * 3, "icnn_width": [32, 32], "load_steps": int(p.load.size),
                "length_scale": 0.02}
    elif name == "notched3d":
        p = I.notched_plate_3d()
        desc = {"workload": "notched_plate_hex8", "elements": p.mesh.n_elems, "qp": p.mesh.n_elems * 8,
                "dofs": p.mesh.n_nodes * 4, "icnn_width": [32, 32], "load_steps": int(p.load.size),
                "length_scale": 0.04}
    elif name == "cube":
        p = I.config3(precision="fp64")
        desc = {"workload": "cube_hex8_64", "elements": p.mesh.n_elems, "qp": p.mesh.n_elems * 8,
                "dofs": p.mesh.n_nodes * 4, "icnn_width": [64, 64], "load_steps": int(p.load.size)}
    else:
        p = I.config1()
        desc = {"workload": "square_q4_8x8", "elements": p.mesh.n_elems, "qp": p.mesh.n_elems * 4,
                "dofs": p.mesh.n_nodes * 3, "icnn_width": [16, 8], "load_steps": int(p.load.size)}
    return p, desc


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
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
            return None
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


def cpu_baseline(prob, seconds, seed=7):
    """The oracle as it stands (single thread): element assembly (residual, tangent,
    local damage update) of a contiguous sample of elements at a seeded state."""
    import numpy as np

    import oracle
    from paper_2604_03411_gb300 import inputs as I
    model = oracle.Model.from_problem(prob)
    rng = np.random.default_rng(seed)
    dofs, kappa = I.random_state(prob.mesh, rng, u_amp=0.02, phi_amp=0.05, kappa_amp=0.02)
    nq = prob.mesh.nq
    t0 = time.perf_counter()
    model.assemble(prob.mesh, dofs, kappa, e0=0, e1=min(64, prob.mesh.n_elems))
    per_elem = (time.perf_counter() - t0) / min(64, prob.mesh.n_elems)
    n = int(max(64, min(prob.mesh.n_elems, seconds / max(per_elem, 1e-9))))
    t0 = time.perf_counter()
    model.assemble(prob.mesh, dofs, kappa, e0=0, e1=n)
    dt = time.perf_counter() - t0
    return {"value": n * nq / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"FP64 oracle assembly (residual, tangent, local damage update) of elements 0..{n - 1} "
                      f"of {prob.mesh.n_elems} ({n * nq} qp) at a seeded state, {dt:.1f} s on 1 host thread"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    prob, desc = make_workload(args.workload)
    if isinstance(prob, list):
        prob = max(prob, key=lambda p: p.mesh.n_elems)
        desc = dict(desc, oracle_sample="largest specimen")
    vals = []
    per_step = max(1.0, 120.0 / max(1, args.steps + args.warmup))
    for k in range(args.warmup + args.steps):
        cb = cpu_baseline(prob, min(per_step, 20.0), seed=100 + k)
        if k >= args.warmup:
            vals.append(cb)
    v = sum(c["value"] for c in vals) / len(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": desc,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": vals[-1]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def mixed_comparison(args, B, torch, prob, batch, stream, flush, reps64, n_qp):
    """The same warm-up and timed load steps in GD_MIXED: device-timed throughput and
    Newton-step time, and the reaction-force error against the FP64 run step by step."""
    import numpy as np
    opts = B.gd_default_options(precision=B.GD_MIXED, cuda_stream=stream.cuda_stream)
    if args.coarse is not None:
        opts.coarse = args.coarse
    h = B.gd_create_batch(prob, opts) if batch else B.gd_create(prob, opts)
    for _ in range(args.warmup):
        B.gd_newton_step(h)
    B.gd_autotune(h)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    reps = []
    reac = []
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record(stream)
        reps.append(B.gd_newton_step(h))
        evs[k][1].record(stream)
        if batch:
            reac.append(None)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    useful = sum(r.iterations + 1 + 2 * r.step_cuts for r in reps)
    r32 = np.array([r.reaction for r in reps])
    r64 = np.array([r.reaction for r in reps64])
    err = float(np.max(np.abs(r32 - r64)) / max(np.max(np.abs(r64)), 1e-300)) if not batch else None
    return {"value": n_qp * useful / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / args.steps,
            "newton_iterations": sum(r.iterations for r in reps),
            "krylov_iterations": sum(r.krylov_iterations for r in reps),
            "krylov_fp32_iterations": sum(r.krylov_fp32_iterations for r in reps),
            "assembly_avg_ms": sum(r.assembly_ms for r in reps) / max(sum(r.assemblies for r in reps), 1),
            "reaction_rel_err_vs_fp64": err,
            "note": "same load steps as the FP64 line; reaction error = max over the timed steps of "
                    "|F_mixed - F_fp64| / max |F_fp64|" if not batch else "batch: per-specimen reactions not compared here"}


def run_gd(args):
    import numpy as np
    import torch

    import paper_2604_03411_gb300.binding as B
    from paper_2604_03411_gb300 import build as build_mod

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build_mod.build()
    prob, desc = make_workload(args.workload, rank, world)
    batch = isinstance(prob, list)
    if args.precision is None:
        args.precision = "mixed" if batch else "fp64"
    stream = torch.cuda.current_stream()
    prec = B.GD_FP64 if args.precision == "fp64" else B.GD_MIXED
    opts = B.gd_default_options(precision=prec, cuda_stream=stream.cuda_stream, inner_solve={"auto": B.GD_INNER_AUTO, "fp64": B.GD_INNER_FP64,
                                             "refined": B.GD_INNER_REFINED}[args.inner])
    if args.coarse is not None:
        opts.coarse = args.coarse
    h = B.gd_create_batch(prob, opts) if batch else B.gd_create(prob, opts)
    coarse_aggs, coarse_n = B.gd_coarse_info(h)
    probs = prob if batch else [prob]
    n_qp = desc["qp"]
    n_path = h.meta["n_steps"]
    n_nodes_all = sum(p.mesh.n_nodes for p in probs)
    n_elems_all = sum(p.mesh.n_elems for p in probs)
    mesh0 = probs[0].mesh
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def step(k):
        if h_state["next"] >= n_path:          # restart the path when it runs out
            B.gd_set_state(h, np.zeros(n_nodes_all * mesh0.ndof), np.zeros((n_elems_all, mesh0.nq)), 0)
            h_state["next"] = 0
        r = B.gd_newton_step(h)
        h_state["next"] += 1
        return r

    h_state = {"next": 0}
    for k in range(args.warmup):
        step(k)
    # launch shapes from the library's own timings at the warmed-up state
    tune = B.gd_autotune(h)
    saved = B.gd_get_state(h)        # the end-to-end leg repeats the timed steps from here
    tuning = {"asm_warps": tune.asm_warps, "krylov_ctas_per_sm": tune.krylov_ctas_per_sm,
              "asm_ms_by_warps": dict(zip(("2", "4", "8"), [round(x, 4) for x in tune.asm_ms])),
              "krylov_us_by_ctas_per_sm": dict(zip(("1", "2", "3", "4"), [round(x, 3) for x in tune.krylov_us])),
              "krylov_node_groups_per_lane": tune.krylov_up,
              "krylov_us_by_node_groups": dict(zip(("1", "2", "4"), [round(x, 3) for x in tune.krylov_us_up]))}
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    reps = []
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()                               # L2 flush between timed steps (outside the events)
        evs[k][0].record(stream)
        reps.append(step(k))
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = sum(a.elapsed_time(b) for a, b in evs)
    asm = sum(r.assemblies for r in reps)
    # qp updates counted per Newton iterate: the first pass of every attempted (sub)step
    # plus the accepted pass of every direction; rejected line-search trials and the
    # mixed mode's FP64 noise pass are work, not progress, and are left out
    useful = sum(r.iterations + 1 + 2 * r.step_cuts for r in reps)
    units = n_qp * useful
    if dist:
        t = torch.tensor([total_ms, float(units)], dtype=torch.float64, device="cuda")
        tm = t.clone()
        dist.all_reduce(tm[0:1], op=dist.ReduceOp.MAX)
        dist.all_reduce(t[1:2], op=dist.ReduceOp.SUM)
        total_ms_all, units_all = float(tm[0]), float(t[1])
    else:
        total_ms_all, units_all = total_ms, float(units)
    value = units_all / (total_ms_all / 1e3)
    newton = sum(r.iterations for r in reps)
    krylov = sum(r.krylov_iterations for r in reps)
    asm_ms = sum(r.assembly_ms for r in reps)
    kry_ms = sum(r.krylov_ms for r in reps)
    launches = sum(r.kernel_launches for r in reps)

    # --- dominant-kernel roofline: persistent Krylov kernel vs the element kernel ---
    # both durations come from CUDA events the library records on its stream around
    # each launch inside the timed steps
    n_dofs = n_nodes_all * mesh0.ndof
    rowptr, colidx = B.gd_csr_pattern(h)
    nnz = colidx.size
    ndof = mesh0.ndof
    peak_bw, peak_kind = measured_peaks()
    asm_avg = asm_ms / max(asm, 1)
    solves = max(newton, 1)
    kry_avg = kry_ms / solves
    iters_per_solve = krylov / solves
    # One BiCGStab iteration (three-barrier form): two SpMVs and the vector phases.
    # Algorithmic bytes: per SpMV the values, the column list once per node block, the
    # row pointers, the gathered x and the written y; the vector phases read/write 25
    # vectors (p, v, y, q, s, t, x~, r, u, rh updates and reads).  Algorithmic FLOPs:
    # 2 per stored value per SpMV, 2 per node-block inverse entry twice, and 2 per
    # element of the 14 vector FMAs / dot products.
    fp32_inner = sum(r.krylov_fp32_iterations for r in reps) * 2 > krylov
    vb = 4 if fp32_inner else 8
    spmv_b = nnz * vb + (nnz // ndof) * 4 + (n_nodes_all + 1) * 4 * 2 + n_dofs * (vb + vb + 1)
    iter_b = 2 * spmv_b + 25 * n_dofs * vb
    iter_f = 2 * (2 * nnz) + 2 * (2 * n_dofs * ndof) + 14 * 2 * n_dofs
    if kry_ms >= asm_ms:
        bytes_launch = iter_b * iters_per_solve
        flops_launch = iter_f * iters_per_solve
        hbm_achieved = bytes_launch / (kry_avg / 1e3) / 1e9
        alu_achieved = flops_launch / (kry_avg / 1e3) / 1e12
        common = {"kernel": "bicgstab3_kernel (persistent Krylov solve of one Newton system)",
                  "avg_launch_ms": kry_avg, "iterations_per_launch": iters_per_solve,
                  "algorithmic_bytes_per_launch": bytes_launch, "algorithmic_flops_per_launch": flops_launch,
                  "traffic_note": "the system (%.0f MB) stays L2-resident across the iterations of a launch, so "
                                  "DRAM traffic is far below the algorithmic bytes" % (spmv_b / 1e6)}
        if fp32_inner:
            roof = dict(common, bound="hbm", achieved=hbm_achieved, peak=peak_bw, unit="GB/s",
                        frac=hbm_achieved / peak_bw, traffic=None, peak_source=f"{peak_kind} copy bandwidth")
        else:
            # FP64 arithmetic issues at 1/64 of the FP32 rate on this part: the FP64 solve is
            # bounded by the FP64 pipe and by its grid barriers, not by memory
            roof = dict(common, bound="alu", achieved=alu_achieved, peak=FP64_PEAK_TFLOPS_NOMINAL, unit="TFLOP/s",
                        frac=alu_achieved / FP64_PEAK_TFLOPS_NOMINAL, traffic=None,
                        peak_source="nominal FP64 rate (1.25 TFLOP/s)",
                        hbm_view={"achieved_gbs": hbm_achieved, "frac_of_measured_copy": hbm_achieved / peak_bw})
    else:
        # element kernel: FP64 (or FP32) ALU bound; algorithmic FLOPs (FMA = 2) of the dense parts
        nq = mesh0.nq
        nd = mesh0.nen * ndof
        evals = sum(r.yield_evals for r in reps)
        # per pass: energy network with tangents at every qp, element tangent; the yield
        # network per local-solve evaluation (qp-weighted mean width over specimens)
        psi_f = sum(p.mesh.n_elems * nq * (10 * p.psi.width ** 2 + 40 * p.psi.width) for p in probs)
        wy = sum(p.mesh.n_elems * p.yld.width for p in probs) / max(n_elems_all, 1)
        flops = asm * psi_f + evals * (4 * wy * wy + 20 * wy) + (asm * n_elems_all) * nd * nd * nq * 25
        achieved = flops / (asm_ms / 1e3) / 1e12
        peak = FP64_PEAK_TFLOPS_NOMINAL if prec == B.GD_FP64 else FP32_PEAK_TFLOPS_NOMINAL
        roof = {"kernel": "element kernel (asm_fp64_kernel)" if prec == B.GD_FP64 else "element kernel (asm_fp32_kernel)",
                "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "peak_source": "nominal FP64 rate" if prec == B.GD_FP64 else
                "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz", "avg_launch_ms": asm_avg,
                "algorithmic_flops_per_launch": flops / max(asm, 1)}

    # --- end to end through the C ABI with host buffers, over the same load steps as
    # the device-timed loop: each step uploads the committed state (dofs, the previous
    # step's dofs for the predictor, kappa) from pinned host memory and reads the new
    # state back ---
    d_np, dp_np, k_np, nxt, dpp_np = saved
    if nxt < 2 or nxt + args.steps > n_path:      # no history to restart from: begin after step 1
        B.gd_set_state(h, np.zeros_like(d_np), np.zeros_like(k_np), 0)
        B.gd_newton_step(h)
        B.gd_newton_step(h)
        d_np, dp_np, k_np, nxt, dpp_np = B.gd_get_state(h)
    d_host = torch.from_numpy(d_np).pin_memory().numpy()
    dp_host = torch.from_numpy(dp_np).pin_memory().numpy()
    dpp_host = torch.from_numpy(dpp_np).pin_memory().numpy()
    k_host = torch.from_numpy(k_np).pin_memory().numpy()
    e2e_ms = 0.0
    e2e_units = 0
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.gd_set_state(h, d_host, k_host, nxt, dofs_prev=dp_host, dofs_prev2=dpp_host)    # host -> device
        r = B.gd_newton_step(h)
        d2, dp2, k2, nxt2, dpp2 = B.gd_get_state(h)                                       # device -> host
        e2e_ms += (time.perf_counter() - t0) * 1e3
        e2e_units += n_qp * (r.iterations + 1 + 2 * r.step_cuts)
        d_host[:], dp_host[:], dpp_host[:], k_host[:], nxt = d2, dp2, dpp2, k2, nxt2
    h2d = d_host.nbytes + dp_host.nbytes + dpp_host.nbytes + k_host.nbytes
    e2e = {"value": e2e_units / (e2e_ms / 1e3) * (world if world > 1 else 1), "unit": UNIT,
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(h2d)}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_all / args.steps, "higher_is_better": True,
        "scaling": "strong" if batch else "weak", "vs_baseline": None,
        "dtype": "f64" if prec == B.GD_FP64 else "f32+f64",
        "data": "synthetic (seeded mesh, seeded ICNN weights)",
        "config": dict(desc, precision=args.precision,
                       parallelism=f"specimen-shards{world}" if batch else f"replicas{world}",
                       inner_solve=args.inner, coarse_unknowns=coarse_n, coarse_aggregates=coarse_aggs,
                       l2="flushed between timed steps (512 MB write)"),
        "newton_step_ms": total_ms / max(newton, 1),
        "newton_iterations": newton, "krylov_iterations": krylov,
        "assembly": {"launches": asm, "counted_passes": useful, "avg_ms": asm_avg,
                     "qp_per_s": n_qp / (asm_avg / 1e3), "share_of_step": asm_ms / total_ms},
        "krylov_share_of_step": kry_ms / total_ms,
        "krylov_ms_per_newton": kry_avg, "krylov_iterations_per_newton": iters_per_solve,
        "krylov_fp32_iterations": sum(r.krylov_fp32_iterations for r in reps),
        "roofline": roof, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk, "tuning": tuning,
    }
    if prec == B.GD_FP64 and not args.no_mixed:
        line["mixed"] = mixed_comparison(args, B, torch, prob, batch, stream, flush, reps, n_qp)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(max(probs, key=lambda p: p.mesh.n_elems), args.cpu_seconds)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_gd(args)


if __name__ == "__main__":
    sys.exit(main())
