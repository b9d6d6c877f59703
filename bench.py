#!/usr/bin/env python3
"""Benchmark of the gradient-enhanced damage hot path on one GB300 per rank.

Metric: qp constitutive+assembly updates/s and Newton-step ms, mixed vs FP64.  One
bench step is one quasi-static load step of the monolithic scheme: Newton
iterations, each an element-kernel pass (kinematics, ICNN energy with derivatives,
yield network and local damage update, degraded stress, residual and consistent
tangent, CSR scatter), the residual norms, the two-level preconditioned BiCGStab
solve and a backtracking line search.  value = (#qp x Newton iterates in the timed
steps) / (timed device time), an iterate being the first pass of a (sub)step or
the accepted pass of a Newton direction: whole-step throughput, inputs resident in
HBM.  Rejected line-search trials are timed but not counted.

Workloads (synthetic, seeded; see paper_2604_03411_gb300/inputs.py):
  cube      3D cube, 64^3 HEX8 (2,097,152 qp), biaxial to lambda = 1.8 in 30 steps,
            both ICNNs width 64; mixed precision with the tensor-core networks
            (default), the same steps in FP64 reported beside it
  notched   2D notched plate 2:1, graded Q4 mesh of 39,936 elements (159,744 qp),
            both ICNNs width 32, 50 steps to 60% nominal strain, FP64 (mixed beside)
  notched3d the paper's thin 3D notched plate, one HEX8 layer of 2,352 elements
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
D_STOP = 0.995                      # damage at which a load path ends (Sec. 5.2)
# FMA throughput measured on this part (a kernel of independent FMA chains, 152 x
# {2, 4, 8} CTAs of 256 threads, timed with CUDA events): FP64 1.19 TFLOP/s, FP32
# 72.8 TFLOP/s.  The copy bandwidth and the BF16 tensor rate come from
# MEASURED_PEAKS.json.
FP64_PEAK_TFLOPS = 1.19
FP32_PEAK_TFLOPS = 72.8
# DRAM traffic of the 3D FP32-vector Krylov kernel with 8 lanes per node, from an ncu capture
# of 40-iteration launches on the 48^3 cube (profiles/krylov_fp32_cube48_traffic.txt): 629 MB
# per iteration against 545 MB of algorithmic bytes.  The capture predates the kernel's
# four-CTA build, so it is not reported as this kernel's traffic (None) until retaken.
KRYLOV_G8_TRAFFIC_PER_ALG = None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gd", choices=["gd", "reference"])
    ap.add_argument("--workload", default="cube", choices=["notched", "notched3d", "cube", "square", "batch"])
    ap.add_argument("--precision", default=None, choices=["fp64", "mixed"],
                    help="default: mixed for the cube and the batch, fp64 otherwise")
    ap.add_argument("--icnn", default="auto", choices=["auto", "cuda", "bf16", "bf16x3"],
                    help="network arithmetic of the mixed element kernel (gd_options.icnn_mma)")
    ap.add_argument("--cube-n", type=int, default=64,
                    help="elements per edge of the cube workload (64 for the bench line; smaller "
                         "cubes for profiler captures)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the other precision's run on the same steps")
    ap.add_argument("--inner", default="auto", choices=["auto", "fp64", "refined"],
                    help="Newton inner-solve policy (gd_options.inner_solve)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--coarse", type=int, default=None,
                    help="coarse unknowns of the two-level preconditioner (gd_options.coarse; 0 = Jacobi only)")
    return ap.parse_args()


def make_workload(name, rank=0, world=1, cube_n=64):
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
        p = I.config3(n=cube_n)
        desc = {"workload": f"cube_hex8_{cube_n}", "elements": p.mesh.n_elems, "qp": p.mesh.n_elems * 8,
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
        return {"hbm_gbs": d.get("hbm_gbs", 6800.0), "bf16_tflops": d.get("bf16_tflops", 1900.0),
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained", 1700.0), "kind": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "kind": "fallback"}


def cpu_baseline(prob, seconds, seed=7, threads=0, single=True):
    """The oracle as it stands: element assembly (residual, tangent, local damage
    update) of a contiguous sample of elements at a seeded state, on all host cores
    (threads=0: the OpenMP default) and, for reference, on one."""
    import numpy as np

    import oracle
    from paper_2604_03411_gb300 import inputs as I
    model = oracle.Model.from_problem(prob)
    rng = np.random.default_rng(seed)
    dofs, kappa = I.random_state(prob.mesh, rng, u_amp=0.02, phi_amp=0.05, kappa_amp=0.02)
    nq = prob.mesh.nq

    def rate(n_threads, secs):
        used = oracle.threads(n_threads)
        n0 = min(4 * used, prob.mesh.n_elems)
        t0 = time.perf_counter()
        model.assemble(prob.mesh, dofs, kappa, e0=0, e1=n0)
        per_elem = (time.perf_counter() - t0) / n0
        n = int(max(n0, min(prob.mesh.n_elems, secs / max(per_elem, 1e-9))))
        t0 = time.perf_counter()
        model.assemble(prob.mesh, dofs, kappa, e0=0, e1=n)
        dt = time.perf_counter() - t0
        return n * nq / dt, n, dt, used

    cores = os.cpu_count() or 1
    va, na, dta, used = rate(threads if threads > 0 else cores, seconds)
    out = {"value": va, "unit": UNIT, "cores": used, "kind": "oracle",
           "sample": f"FP64 oracle assembly (residual, tangent, local damage update) of elements 0..{na - 1} "
                     f"of {prob.mesh.n_elems} ({na * nq} qp) at a seeded state, {dta:.1f} s on {used} host threads"}
    if single:
        v1, n1, dt1, _ = rate(1, seconds / 3.0)
        out["single_thread_value"] = v1
        out["sample"] += f"; one thread: {n1} elements in {dt1:.1f} s"
    oracle.threads(cores)
    return out


def run_config(args, desc, batch, world):
    """The workload's configuration as both arms report it (no measured quantities)."""
    precision = args.precision or ("mixed" if (batch or args.workload == "cube") else "fp64")
    icnn = args.icnn if args.icnn != "auto" else ("cuda" if batch else "bf16x3")
    return dict(desc, precision=precision, icnn_mma=icnn if precision == "mixed" else None,
                parallelism=f"specimen-shards{world}" if batch else f"replicas{world}",
                inner_solve=args.inner, l2="flushed between timed steps (512 MB write)",
                path_end=f"restart from the undeformed state when the path runs out or max damage >= {D_STOP}")


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return 0
    prob, desc = make_workload(args.workload, cube_n=args.cube_n)
    batch = isinstance(prob, list)
    config = run_config(args, desc, batch, world)
    if batch:
        prob = max(prob, key=lambda p: p.mesh.n_elems)
    vals = []
    per_step = max(1.0, 120.0 / max(1, args.steps + args.warmup))
    for k in range(args.warmup + args.steps):
        cb = cpu_baseline(prob, min(per_step, 20.0), seed=100 + k, single=False)
        if k >= args.warmup:
            vals.append(cb)
    v = sum(c["value"] for c in vals) / len(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[-1]["cores"], "kind": "oracle",
                             "sample": vals[-1]["sample"] + (" (the largest specimen)" if batch else "")},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


ICNN = {"auto": 0, "cuda": 1, "bf16": 2, "bf16x3": 3}


def krylov_roofline(reps, nnz, n_dofs, n_nodes, ndof, kry_ms, peaks, fp32_inner, lanes=0):
    """Algorithmic bytes and FLOPs of the persistent Krylov launches (one per Newton
    system).  One BiCGStab iteration (three-barrier form): two products with the
    values, the column list once per node block, the row pointers, the gathered x
    and the written y; the vector phases read and write 25 vectors.  FLOPs: 2 per
    stored value per product, the node-block inverse twice, 14 vector FMAs / dots."""
    newton = max(sum(r.iterations for r in reps), 1)
    krylov = sum(r.krylov_iterations for r in reps)
    vb = 4 if fp32_inner else 8
    spmv_b = nnz * vb + (nnz // ndof) * 4 + (n_nodes + 1) * 4 * 2 + n_dofs * (vb + vb + 1)
    iter_b = 2 * spmv_b + 25 * n_dofs * vb
    iter_f = 2 * (2 * nnz) + 2 * (2 * n_dofs * ndof) + 14 * 2 * n_dofs
    avg = kry_ms / newton
    ipl = krylov / newton
    hbm = iter_b * ipl / (avg / 1e3) / 1e9
    alu = iter_f * ipl / (avg / 1e3) / 1e12
    common = {"kernel": "bicgstab3_kernel (persistent two-level BiCGStab, one launch per Newton system)",
              "avg_launch_ms": avg, "iterations_per_launch": ipl, "us_per_iteration": 1e3 * avg / max(ipl, 1e-9),
              "algorithmic_bytes_per_launch": iter_b * ipl, "algorithmic_flops_per_launch": iter_f * ipl,
              "bytes_per_iteration": iter_b}
    if fp32_inner or iter_b > 129e6:
        traffic = None
        if KRYLOV_G8_TRAFFIC_PER_ALG and fp32_inner and ndof == 4 and lanes == 8:
            traffic = KRYLOV_G8_TRAFFIC_PER_ALG * iter_b * ipl
            common["traffic_source"] = ("ncu dram bytes of the 8-lane FP32 kernel on the 48^3 cube, "
                                        "scaled by algorithmic bytes")
        return dict(common, bound="hbm", achieved=hbm, peak=peaks["hbm_gbs"], unit="GB/s",
                    frac=hbm / peaks["hbm_gbs"], traffic=traffic, peak_source=f"{peaks['kind']} copy bandwidth",
                    alu_view={"achieved_tflops": alu, "fp64_peak": FP64_PEAK_TFLOPS})
    return dict(common, bound="alu", achieved=alu, peak=FP64_PEAK_TFLOPS, unit="TFLOP/s",
                frac=alu / FP64_PEAK_TFLOPS, traffic=None, peak_source="measured FP64 FMA rate",
                hbm_view={"achieved_gbs": hbm, "frac_of_copy": hbm / peaks["hbm_gbs"]},
                note="the system stays L2-resident across the iterations of a launch")


def element_roofline(reps, probs, n_elems_all, fp64, icnn, peaks):
    """Counted algorithmic FLOPs of the element kernel per launch: the energy network
    with its forward tangents and reverse column (10 w^2 + 40 w per point), the
    yield network per local-solve evaluation (4 w^2 + 20 w), the element tangent
    (25 nd^2 per point).  The networks' second layers (8 w^2 + 2 w^2 per point,
    4 w^2 per evaluation) run on the tensor cores in the BF16 modes."""
    asm = max(sum(r.assemblies for r in reps), 1)
    asm_ms = sum(r.assembly_ms for r in reps)
    mesh0 = probs[0].mesh
    nq, nd = mesh0.nq, mesh0.nen * mesh0.ndof
    evals = sum(r.yield_evals for r in reps)
    qp_all = sum(p.mesh.n_elems * nq for p in probs)
    psi_f = sum(p.mesh.n_elems * nq * (10 * p.psi.width ** 2 + 40 * p.psi.width) for p in probs)
    psi_mma = sum(p.mesh.n_elems * nq * 10 * p.psi.width ** 2 for p in probs)
    wy = sum(p.mesh.n_elems * p.yld.width for p in probs) / max(n_elems_all, 1)
    flops = asm * psi_f + evals * (4 * wy * wy + 20 * wy) + asm * n_elems_all * nd * nd * nq * 25
    mma = asm * psi_mma + evals * 4 * wy * wy
    t = asm_ms / 1e3
    avg = asm_ms / asm
    if fp64:
        return {"kernel": "asm_fp64_kernel", "bound": "alu", "achieved": flops / t / 1e12, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": flops / t / 1e12 / FP64_PEAK_TFLOPS, "traffic": None,
                "peak_source": "measured FP64 FMA rate", "avg_launch_ms": avg,
                "algorithmic_flops_per_launch": flops / asm, "qp_per_launch": qp_all}
    tc = icnn in ("bf16", "bf16x3")
    cuda_f = flops - (mma if tc else 0)
    out = {"kernel": "asm_tc_kernel" if tc else "asm_fp32_kernel", "bound": "alu",
           "achieved": cuda_f / t / 1e12, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
           "frac": cuda_f / t / 1e12 / FP32_PEAK_TFLOPS, "traffic": None, "peak_source": "measured FP32 FMA rate",
           "avg_launch_ms": avg, "algorithmic_flops_per_launch": flops / asm, "qp_per_launch": qp_all,
           "note": "FLOPs on the CUDA cores (network layer 1 and epilogues, local solve, tangent rows)"}
    if tc:
        prod = 3 if icnn == "bf16x3" else 1
        out["tensor_view"] = {"mma_flops_per_launch": mma / asm, "tensor_products": prod,
                              "achieved_tflops": prod * mma / t / 1e12,
                              "frac_of_bf16_peak": prod * mma / t / 1e12 / peaks["bf16_tflops_sustained"],
                              "peak_source": f"{peaks['kind']} BF16 dense (sustained)"}
    return out


def timed_run(args, B, torch, probs, batch, precision, stream, flush, n_path, steps, warmup, tune=True,
              schedule=None):
    """W untimed load steps, gd_autotune, then K steps timed with CUDA events on the
    library's stream, the L2 flushed between them.  Returns the handle, the reports,
    the timings, the saved state, the tuning, the step function and the restart
    schedule (one flag per warm-up and timed step: the path restarted before it).
    schedule: restart flags to follow instead of deciding (the other precision then
    runs exactly the same load steps)."""
    import numpy as np
    prec = B.GD_FP64 if precision == "fp64" else B.GD_MIXED
    opts = B.gd_default_options(precision=prec, cuda_stream=stream.cuda_stream,
                                inner_solve={"auto": B.GD_INNER_AUTO, "fp64": B.GD_INNER_FP64,
                                             "refined": B.GD_INNER_REFINED}[args.inner],
                                icnn_mma=ICNN[args.icnn])
    if args.coarse is not None:
        opts.coarse = args.coarse
    h = B.gd_create_batch(probs, opts) if batch else B.gd_create(probs[0], opts)
    n_nodes_all = sum(p.mesh.n_nodes for p in probs)
    n_elems_all = sum(p.mesh.n_elems for p in probs)
    mesh0 = probs[0].mesh
    state = {"next": 0, "dmax": 0.0, "k": 0}
    flags = []

    def step():
        # the path restarts from the undeformed state when it runs out or once a step
        # has brought the largest damage to D_STOP (the uniform-deformation runs of
        # Sec. 5.2 stop there: beyond it the block carries no load and the steps only
        # probe a vanishing stiffness)
        k = state["k"]
        state["k"] += 1
        if schedule is not None and k < len(schedule):
            restart = schedule[k]
        else:
            restart = state["next"] >= n_path or state["dmax"] >= D_STOP
        flags.append(bool(restart))
        if restart:
            B.gd_set_state(h, np.zeros(n_nodes_all * mesh0.ndof), np.zeros((n_elems_all, mesh0.nq)), 0)
            state["next"] = 0
        r = B.gd_newton_step(h)
        state["next"] += 1
        state["dmax"] = r.max_damage
        return r

    for _ in range(warmup):
        step()
    tuning = None
    if tune:
        t = B.gd_autotune(h)
        tuning = {"asm_warps": t.asm_warps, "krylov_ctas_per_sm": t.krylov_ctas_per_sm,
                  "asm_ms_by_warps": dict(zip(("2", "4", "8"), [round(x, 4) for x in t.asm_ms])),
                  "krylov_us_by_ctas_per_sm": dict(zip(("1", "2", "3", "4"), [round(x, 3) for x in t.krylov_us])),
                  "krylov_node_groups_per_lane": t.krylov_up,
                  "krylov_us_by_node_groups": dict(zip(("1", "2", "4"), [round(x, 3) for x in t.krylov_us_up])),
                  "krylov_lanes_per_node": t.krylov_lanes,
                  "krylov_us_by_lanes": dict(zip(("32", "8", "4"), [round(x, 3) for x in t.krylov_us_lanes]))}
    saved = (B.gd_get_state(h), state["dmax"])
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    reps = []
    for k in range(steps):
        flush.zero_()                               # L2 flush between timed steps (outside the events)
        evs[k][0].record(stream)
        reps.append(step())
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    total_ms = sum(a.elapsed_time(b) for a, b in evs)
    return h, reps, total_ms, saved, tuning, step, list(flags)


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
    prob, desc = make_workload(args.workload, rank, world, cube_n=args.cube_n)
    batch = isinstance(prob, list)
    probs = prob if batch else [prob]
    if args.precision is None:
        args.precision = "mixed" if (batch or args.workload == "cube") else "fp64"
    # network arithmetic of the mixed runs (auto: tensor-core BF16x3 for one specimen)
    icnn = args.icnn if args.icnn != "auto" else ("cuda" if batch else "bf16x3")
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    n_path = max(int(p.load.size) for p in probs)
    n_qp = desc["qp"]
    n_nodes_all = sum(p.mesh.n_nodes for p in probs)
    n_elems_all = sum(p.mesh.n_elems for p in probs)
    mesh0 = probs[0].mesh
    ndof = mesh0.ndof
    peaks = measured_peaks()

    if dist:
        dist.barrier()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    h, reps, total_ms, saved, tuning, step, sched = timed_run(args, B, torch, probs, batch, args.precision, stream,
                                                             flush,
                                                      n_path, args.steps, args.warmup)
    clk = clocks.stop()
    coarse_aggs, coarse_n = B.gd_coarse_info(h)
    nnz = B.gd_csr_pattern(h)[1].size
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

    def summary(reps, total_ms, precision):
        newton = sum(r.iterations for r in reps)
        krylov = sum(r.krylov_iterations for r in reps)
        asm = sum(r.assemblies for r in reps)
        asm_ms = sum(r.assembly_ms for r in reps)
        kry_ms = sum(r.krylov_ms for r in reps)
        fp32_inner = sum(r.krylov_fp32_iterations for r in reps) * 2 > krylov
        lanes = (tuning or {}).get("krylov_lanes_per_node", 0) if precision == args.precision else 0
        kroof = krylov_roofline(reps, nnz, n_nodes_all * ndof, n_nodes_all, ndof, kry_ms, peaks, fp32_inner, lanes)
        eroof = element_roofline(reps, probs, n_elems_all, precision == "fp64", icnn, peaks)
        dominant = kroof if kry_ms >= asm_ms else eroof
        return {"newton_step_ms": total_ms / max(newton, 1), "newton_iterations": newton,
                "krylov_iterations": krylov, "krylov_fp32_iterations": sum(r.krylov_fp32_iterations for r in reps),
                "assembly": {"launches": asm, "avg_ms": asm_ms / max(asm, 1),
                             "qp_per_s": n_qp / (asm_ms / max(asm, 1) / 1e3), "share_of_step": asm_ms / total_ms},
                "krylov_share_of_step": kry_ms / total_ms, "krylov_ms_per_newton": kry_ms / max(newton, 1),
                "krylov_iterations_per_newton": krylov / max(newton, 1),
                "step_cuts": sum(r.step_cuts for r in reps), "gpu_launches": int(sum(r.kernel_launches for r in reps)),
                "roofline": dominant, "roofline_kernels": {"element": eroof, "krylov": kroof}}

    main = summary(reps, total_ms, args.precision)

    # --- end to end through the C ABI with host buffers, over the same load steps as
    # the device-timed loop: each step uploads the committed state (dofs, the two
    # previous states for the predictor, kappa) from pinned host memory and reads the
    # new state back ---
    (d_np, dp_np, k_np, nxt, dpp_np), dmax = saved
    d_host = torch.from_numpy(d_np).pin_memory().numpy()
    dp_host = torch.from_numpy(dp_np).pin_memory().numpy()
    dpp_host = torch.from_numpy(dpp_np).pin_memory().numpy()
    k_host = torch.from_numpy(k_np).pin_memory().numpy()
    e2e_ms = 0.0
    e2e_units = 0
    for k in range(args.steps):
        flush.zero_()
        kk = args.warmup + k
        restart = sched[kk] if kk < len(sched) else (nxt >= n_path or dmax >= D_STOP)
        if restart:                                # the path's end, as in the timed loop
            d_host[:] = 0.0
            k_host[:] = 0.0
            nxt = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if nxt >= 2:                               # host -> device: the state and the predictor's history
            B.gd_set_state(h, d_host, k_host, nxt, dofs_prev=dp_host, dofs_prev2=dpp_host)
        elif nxt == 1:
            B.gd_set_state(h, d_host, k_host, nxt, dofs_prev=dp_host)
        else:
            B.gd_set_state(h, d_host, k_host, nxt)
        r = B.gd_newton_step(h)
        d2, dp2, k2, nxt2, dpp2 = B.gd_get_state(h)                                       # device -> host
        e2e_ms += (time.perf_counter() - t0) * 1e3
        e2e_units += n_qp * (r.iterations + 1 + 2 * r.step_cuts)
        d_host[:], dp_host[:], dpp_host[:], k_host[:], nxt = d2, dp2, dpp2, k2, nxt2
        dmax = r.max_damage
    h2d = d_host.nbytes + dp_host.nbytes + dpp_host.nbytes + k_host.nbytes
    e2e = {"value": e2e_units / (e2e_ms / 1e3) * (world if world > 1 else 1), "unit": UNIT,
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(h2d)}
    del h

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_all / args.steps, "higher_is_better": True,
        "scaling": "strong" if batch else "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else ("bf16x3+f32+f64" if icnn == "bf16x3" else
                                                         "bf16+f32+f64" if icnn == "bf16" else "f32+f64"),
        "data": "synthetic (seeded mesh, seeded ICNN weights)",
        "config": run_config(args, desc, batch, world),
        "coarse": {"unknowns": coarse_n, "aggregates": coarse_aggs},
    }
    line.update({k: v for k, v in main.items() if k != "gpu_launches"})
    line["e2e"] = e2e
    line["gpu_launches"] = main["gpu_launches"]
    line["clocks"] = clk
    line["tuning"] = tuning
    # --- the other precision over the same load steps ---
    if not args.no_compare:
        other = "fp64" if args.precision == "mixed" else "mixed"
        # the same load steps: the restarts follow the first run's schedule
        h2, reps2, ms2, _, _, _, _ = timed_run(args, B, torch, probs, batch, other, stream, flush, n_path, args.steps,
                                               args.warmup, tune=True, schedule=sched)
        useful2 = sum(r.iterations + 1 + 2 * r.step_cuts for r in reps2)
        sub = {"value": n_qp * useful2 / (ms2 / 1e3), "unit": UNIT, "ms_per_step": ms2 / args.steps}
        sub.update(summary(reps2, ms2, other))
        if not batch:
            r_mixed = np.array([r.reaction for r in (reps if args.precision == "mixed" else reps2)])
            r_fp64 = np.array([r.reaction for r in (reps2 if args.precision == "mixed" else reps)])
            scale = max(np.max(np.abs(r_fp64)), 1e-300)
            line["reaction_rel_err_mixed_vs_fp64"] = float(np.max(np.abs(r_mixed - r_fp64)) / scale)
            # by the damage the step reached: near d = 1 the reaction is a few percent of
            # its peak and the mixed residual's rounding floor decides its last digits
            dmx = np.array([r.max_damage for r in (reps2 if args.precision == "mixed" else reps)])
            bins = {}
            for name, lo, hi in (("d<0.9", -1.0, 0.9), ("0.9<=d<0.99", 0.9, 0.99), ("d>=0.99", 0.99, 2.0)):
                sel = (dmx >= lo) & (dmx < hi)
                if sel.any():
                    bins[name] = {"steps": int(sel.sum()),
                                  "of_peak": float(np.max(np.abs(r_mixed - r_fp64)[sel]) / scale),
                                  "of_step": float(np.max(np.abs(r_mixed - r_fp64)[sel] /
                                                          np.maximum(np.abs(r_fp64[sel]), 1e-300)))}
            line["reaction_err_by_damage"] = bins
        line[other] = sub
        line["speedup_mixed_over_fp64"] = (value / sub["value"]) if args.precision == "mixed" else (sub["value"] / value)
        del h2
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
