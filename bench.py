"""Benchmark of the fused BEM assembly + Rayleigh-Ritz projection on one GB300 per rank.

One step is one pass of the hot path over the largest single-GPU workload, the ellipsoid
of semi-axes (1.0, 0.7, 0.5) meshed by 98304 flat triangles (circle contour centre 9.0,
radius 1.5, N = 64 trapezoid nodes; Ritz basis of 256 complex Gaussian columns; near
panel pairs by the 8 x 8 rule):
  geometry set-up -> contour nodes, weights and self terms -> CholeskyQR2 of the basis ->
  fused assembly + projection Bhat_j = w_j V^H A(z_j) V for all 64 nodes.
The metric counts n^2 N matrix entries assembled and projected per step. The accuracy
qualifier (untimed) solves the eigenproblem from the same basis (Algorithm 1, CholeskyQR2,
mixed projection, reduced solve, refinement) and reports every eigenpair inside the
contour with its FP64 residual; where the oracle's eigenvalues are stored (tests/golden)
it also compares against them.

``--workload`` selects another of the synthetic workloads for a separate line:
``cube3072`` (unit cube, 16 x 16 squares per face, ellipse centre 6.5 semi-axes 1.5 and
0.4, N = 32, nu = 64), ``sphere20480`` (icosphere level 5, circle centre 7 radius 1,
N = 32, nu = 128; ``--near`` 0/1/2 selects no near-field treatment, the 8 x 8 rule, or the
surrogate network, trained beforehand, untimed), ``batch48`` (48 ellipsoids of uneven size
through the grouped persistent launch replayed as a CUDA graph; a step is one replay) and
``ellipsoid24576`` (the level-5 mesh of the default ellipsoid, N = 16: a small case of the
same kernel shape for profiler captures).

Ranks (torchrun) run independent replicas of the step (the path has no exchange step) and
the reported value is the sum over ranks (weak scaling). ``--impl reference`` times the
CPU FP64 oracle on a bounded row sample of the same workload instead (rank 0 only).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BEM entries assembled+projected/s at eig rel err ≤1e-8; % of roofline"
UNIT = "entries/s"
WORKLOAD = "ellipsoid98304"
L2_FLUSH_BYTES = 512 << 20   # > 129 MB L2


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="mixed", choices=["fp64", "mixed", "hmatrix"])
    p.add_argument("--plain-steps", type=int, default=2,
                   help="steps of the plain FP64 path timed for the speedup (0: skip)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-eig-check", action="store_true")
    p.add_argument("--workload", default=WORKLOAD,
                   choices=["cube3072", "sphere20480", "ellipsoid98304", "batch48",
                            "ellipsoid24576"])
    p.add_argument("--near", type=int, default=None, choices=[0, 1, 2],
                   help="near-field mode (default: 1 for sphere20480 and ellipsoid98304, else 0)")
    p.add_argument("--operator", default="single", choices=["single", "neumann", "robin"],
                   help="boundary operator: single layer (default), double layer with its jump "
                        "(Neumann), or Robin 0.5 G + (1/2 I + K)")
    p.add_argument("--twin-clusters", type=int, default=1, choices=[0, 1],
                   help="units of one node (nu > 128): twin pairs on two-CTA clusters (1, "
                        "default) or one node per CTA (0)")
    p.add_argument("--sweep-eval-split", action="store_true",
                   help="instead of the projection bench: time the fused kernel at every split "
                        "of its sines and cosines between the MUFU unit and the FMA-pipe "
                        "polynomials (0..4 of the 7 quadrature points), with the pipe rates")
    p.add_argument("--inverse-power", type=int, default=0, metavar="Q",
                   help="instead of the projection bench: time Q steps of Algorithm 1 on the "
                        "workload, dense (FP32 LU of S) against matrix-free (GMRES)")
    return p.parse_args()


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

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
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def problem(name=WORKLOAD):
    import synth
    prob = synth.workload(name).problems[0]
    mesh = prob.mesh()
    V = synth.complex_gaussian(mesh.n, prob.nu, prob.seed)
    return prob, mesh, V


def oracle_sample(prob, mesh, V, target_s=12.0):
    """Times the oracle's assembly + projection on a row sample sized to ~target_s."""
    import oracle
    from oracle import contour as ocon, rr as orr
    oracle.build()
    z, w = ocon.from_spec(prob.contour, prob.N)
    rows = 16
    while True:
        t0 = time.perf_counter()
        orr.project(mesh, z, V, rows=(0, rows))
        dt = time.perf_counter() - t0
        if dt >= target_s or rows >= mesh.n:
            break
        rows = min(mesh.n, max(2 * rows, int(rows * target_s / max(dt, 1e-3))))
    entries = rows * mesh.n * prob.N
    cores = oracle.lib().oracle_max_threads()
    return {"value": entries / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "seconds": dt,
            "sample": f"rows 0..{rows} of {mesh.n} (all {mesh.n} columns, all {prob.N} "
                      f"nodes, nu={prob.nu}): {entries:.3e} entries in {dt:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    prob, mesh, V = problem(args.workload if args.workload != "batch48" else WORKLOAD)
    times, secs = [], []
    base = None
    for it in range(args.warmup + args.steps):
        b = oracle_sample(prob, mesh, V, target_s=8.0 if it >= args.warmup else 1.0)
        if it >= args.warmup:
            times.append(b["value"])
            secs.append(b["seconds"])
            base = b
    value = statistics.median(times)
    # a step is one bounded sample of the workload (its rows are named in config.sample)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.median(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload if args.workload != "batch48" else WORKLOAD,
                       "n": mesh.n, "N": prob.N, "nu": prob.nu, "sample": base["sample"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": base["cores"],
                             "kind": "oracle", "sample": base["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def unit_nodes(N, nu, cap):
    """Nodes per work unit of the mixed kernel: up to 4 (or the cap), within the 512 TMEM
    accumulator columns (2 nup per node, nup = nu rounded up to 8, above 128 to 128)."""
    nup = (nu + 7) // 8 * 8
    if nup > 128:
        nup = (nup + 127) // 128 * 128
    g = min(N, min(cap, 4) if cap > 0 else 4)
    return max(1, min(g, 512 // (2 * nup)))


def mufu_seconds_per_entry(rates, N, G, twins, clusters=False):
    """MUFU time of one entry of A for all N nodes at the measured rates: per quadrature
    point (7) one ex2 per node, one sin and one cos per node or per twin pair evaluated
    together (the pair in one unit, starting at an even slot), one rsqrt per unit.
    clusters: units of one node whose twin pairs run on two-CTA clusters, each entry of a
    pair evaluated once for both nodes (one rsqrt, sin and cos per pair)."""
    if clusters:
        phases = N - twins
        return 7 * (N / rates["ex2"] + phases * (1 / rates["sin"] + 1 / rates["cos"] +
                                                 1 / rates["rsqrt"]))
    paired = 0
    for P in range(twins):
        s0 = 2 * P
        if s0 // G == (s0 + 1) // G and (s0 // G * G) % 2 == 0:
            paired += 1
    phases = N - paired
    units = -(-N // G)
    return 7 * (N / rates["ex2"] + phases * (1 / rates["sin"] + 1 / rates["cos"]) +
                units / rates["rsqrt"])


def mufu_seconds_method(rates, N):
    """The method's own evaluation work per entry for all N nodes, at the measured rates:
    7 quadrature points, each one complex exponential per node (ex2, sin, cos) and one
    rsqrt shared by all N nodes; no work shared between nodes beyond that."""
    return 7 * (N * (1 / rates["ex2"] + 1 / rates["sin"] + 1 / rates["cos"]) + 1 / rates["rsqrt"])


def measured_traffic(workload, precision):
    """DRAM bytes (read + write) per launch of the dominant kernel (the fused kernel, or the
    far field's leaf kernel) from the committed ncu summary of this workload, or None when
    there is none or the kernel's source has changed since the counters were taken (the
    summary records the source's SHA-256)."""
    import hashlib
    names = {"mixed": ("mixed_apply", "project_mixed.cu"), "hmatrix": ("hm_leaf", "hmatrix.cu")}
    if precision not in names:
        return None
    kernel, source = names[precision]
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    src = os.path.join(ROOT, "paper_1906_03938_gb300", "csrc", source)
    with open(src, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    if rec.get("source_sha256") != sha:
        return None
    return rec["dram_bytes_read"] + rec["dram_bytes_write"]


def read_golden(name):
    """(eigenvalue, multiplicity) of the stored oracle eigenvalues of a workload that lie
    inside its contour, or None when the workload has no stored list."""
    path = os.path.join(ROOT, "tests", "golden", f"eigs_{name}.txt")
    if not os.path.exists(path):
        return None
    gold = []
    for line in open(path):
        if not line.startswith("#"):
            re_, im_, mult, ins = line.split()
            if int(ins):
                gold.append((complex(float(re_), float(im_)), int(mult)))
    return gold


def inside_contour(lam, spec, margin=0.0):
    """True where lam lies inside the ellipse (circle) of ``spec`` shrunk by ``margin``."""
    lam = np.asarray(lam)
    x = (lam.real - spec.centre.real) / spec.a
    y = (lam.imag - spec.centre.imag) / spec.b
    return np.sqrt(x * x + y * y) < 1.0 - margin


def eig_compare(lam, X, rel, gold, spec, tol, conv=1e-10, margin=0.02):
    """Compares a solve's eigenpairs (lam, columns of X, relative residuals rel) with the
    expected list ``gold`` of (eigenvalue, multiplicity) inside the contour:
      * every expected eigenvalue has a found value within tol (relative) whose residual is
        below conv, and at least its multiplicity of independent vectors there (missing);
      * every converged value (rel < conv) strictly inside the contour (shrunk by the
        relative margin; the annulus next to the contour may hold values either way) is
        within tol of an expected one (extras).
    Returns a dict with the per-eigenvalue errors and residuals, the missing and extra
    values and ``ok``."""
    lam = np.asarray(lam, dtype=np.complex128)
    rel = np.asarray(rel, dtype=np.float64)
    Xh = np.asarray(X)
    per, missing = [], []
    for g, m in gold:
        near = np.where((np.abs(lam - g) <= tol * abs(g)) & (rel < conv))[0]
        err = float(np.min(np.abs(lam - g)) / abs(g)) if len(lam) else float("inf")
        rank = 0
        if len(near):
            cols = Xh[:, near] / np.linalg.norm(Xh[:, near], axis=0)
            rank = int(np.sum(np.linalg.svd(cols, compute_uv=False) > 1e-6))
        rr = float(np.max(rel[near])) if len(near) else None
        per.append({"expected": [g.real, g.imag], "multiplicity": m, "rel_err": err,
                    "relres_max": rr, "vectors": rank})
        if len(near) == 0 or rank < m:
            missing.append([g.real, g.imag, m, rank])
    extras = []
    for k in np.where((rel < conv) & inside_contour(lam, spec, margin))[0]:
        if not any(abs(lam[k] - g) <= tol * abs(g) for g, _ in gold):
            extras.append([lam[k].real, lam[k].imag, float(rel[k])])
    errs = [p["rel_err"] for p in per]
    return {"ok": not missing and not extras, "per_eigenvalue": per, "missing": missing,
            "extras": extras, "eig_rel_err_max": max(errs) if errs else None,
            "relres_max": float(np.max(rel)) if len(rel) else None,
            "multiplicities_ok": not missing}


def train_surrogate(bem, device, epochs=200):
    """Training data from the near pairs of two spheres and an ellipsoid (k over the
    contours' range), then training with the library's own kernels; returns the parameters
    and the loss history."""
    import torch
    import synth
    t0 = time.perf_counter()
    feats, targs = [], []
    for seed, mesh in ((21, synth.icosphere(3)), (22, synth.icosphere(4)),
                       (23, synth.tetrakis_sphere(3, (1.0, 0.7, 0.5)))):
        c = bem.Context(device)
        c.set_mesh(mesh.xyz, mesh.tri)
        c.set_near_field(1)
        # Re k from 2.5: the training meshes' panels are 2-4x the workload's, so k h of the
        # workload's pairs (k on the contour) lies inside the box this range spans
        f, t = c.surrogate_samples(300000, (2.5, 10.5), (-1.5, 1.5), seed=seed)
        feats.append(f)
        targs.append(t)
        c.close()
    feat, targ = torch.cat(feats), torch.cat(targs)
    tr = bem.Context(device)
    tr.surrogate_init(seed=5)
    losses = tr.surrogate_train(feat, targ, epochs=epochs, batch=4096, lr=3e-3)
    params = tr.surrogate_params(which=0)
    tr.close()
    return {"params": params, "samples": int(feat.shape[0]), "epochs": epochs,
            "loss_first": float(losses[0]), "loss_last": float(losses[-1]),
            "train_s": time.perf_counter() - t0}


def run_batch(args):
    """The 48-ellipsoid sweep through the grouped persistent launch (CUDA graph)."""
    import torch
    import paper_1906_03938_gb300 as bem
    import synth
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1906_03938_gb300.sharding import rank_share
    probs_all = synth.workload("batch48").problems
    meshes_all = [p.mesh() for p in probs_all]
    costs = [float(m.n) * m.n * p.N for m, p in zip(meshes_all, probs_all)]
    # independent problems: each rank takes its share by work, no data exchange
    mine = rank_share(costs, rank, world)
    probs = [probs_all[i] for i in mine]
    ctxs, Vh, Vd, meshes = [], [], [], []
    for i_prob, prob in zip(mine, probs):
        mesh = meshes_all[i_prob]
        c = bem.Context(local)
        c.set_mesh(mesh.xyz, mesh.tri)
        c.set_contour(prob.contour.kind, prob.contour.centre, prob.contour.a, prob.contour.b, prob.N)
        V = synth.complex_gaussian(mesh.n, prob.nu, prob.seed)
        Vh.append(torch.from_numpy(np.asfortranarray(V)).pin_memory())
        Vd.append(bem.fortran(Vh[-1].to(dev)))
        ctxs.append(c)
        meshes.append(mesh)
    t0 = time.perf_counter()
    batch = bem.Batch(ctxs, Vd, autotune=True)
    tune_s = time.perf_counter() - t0
    info = batch.info()
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        batch.run()
    torch.cuda.synchronize()
    launches0 = sum(c.launches for c in ctxs)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        batch.run()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_total = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    launches = sum(c.launches for c in ctxs) - launches0
    # end to end: host bases in, projected matrices out, every step
    Bh = [torch.empty(B.shape, dtype=B.dtype).pin_memory() for B in batch.Bhat]
    e2e = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(float(k))
        e2e[k][0].record(stream)
        for a, b in zip(Vd, Vh):
            a.copy_(b, non_blocking=True)
        batch.run()
        for a, b in zip(Bh, batch.Bhat):
            a.copy_(b, non_blocking=True)
        e2e[k][1].record(stream)
    torch.cuda.synchronize()
    e2e_total = sum(a.elapsed_time(b) for a, b in e2e) / 1e3
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([t_total, e2e_total], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_total, e2e_total = float(t[0]), float(t[1])
    entries = float(sum(costs))          # all problems of all ranks
    value = entries * args.steps / t_total
    if rank != 0:
        return 0
    rates = {k: ctxs[0].microbench(k) for k in ("ex2", "sin", "cos", "rsqrt")}
    step_s = t_total / args.steps
    mine_entries = float(sum(costs[i] for i in mine))
    # MUFU seconds of this rank's work: each problem at its own node count, schedule and
    # nodes per unit (the batch's cap, else 4, within the accumulator limit)
    t_mufu = 0.0
    for k, i in enumerate(mine):
        Nk = probs_all[i].N
        Gk = unit_nodes(Nk, probs_all[i].nu, batch.info()["nodes_per_unit"])
        t_mufu += costs[i] / Nk * mufu_seconds_per_entry(rates, Nk, Gk, ctxs[k].node_order()[1])
    t_entry = t_mufu / mine_entries
    roof = {"bound": "alu", "pipe": "mufu", "achieved": mine_entries / step_s, "peak": 1.0 / t_entry,
            "unit": "entries/s", "frac": mine_entries / step_s * t_entry, "traffic": None,
            "kernel_ms": 1e3 * step_s,
            "peak_source": "measured MUFU rates (bem_microbench); achieved over the whole graph "
                           "replay (preparation, grouped kernel, reductions), not the kernel alone"}
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = oracle_sample(probs[0], meshes[0], synth.complex_gaussian(meshes[0].n, probs[0].nu,
                                                                        probs[0].seed))
    # accuracy qualifier (untimed): every problem of this rank solved from its own basis
    # (Algorithm 1, CholeskyQR2, mixed projection, reduced solve, refinement), each
    # eigenpair with its FP64 residual; problems with stored oracle eigenvalues compared
    eig = None
    if not args.no_eig_check:
        t0 = time.perf_counter()
        per = []
        for k, i_prob in enumerate(mine):
            spec = probs_all[i_prob].contour
            r = eig_check(ctxs[k], Vd[k], bem.PREC_MIXED, spec, read_golden(f"batch48_p{i_prob}"),
                          "mixed")
            entry = {"problem": i_prob, "n": meshes[k].n, "N": probs_all[i_prob].N,
                     "centre": spec.centre.real, "found": len(r.get("found", [])),
                     "converged": r.get("converged_inside"),
                     "relres_max_converged": r.get("relres_max_converged"),
                     "solve_s": r.get("solve_s")}
            if "error" in r:
                entry["error"] = r["error"]
            if "ok" in r:
                entry.update({"golden_ok": r["ok"], "eig_rel_err_max": r["eig_rel_err_max"],
                              "missing": r["missing"], "extras": r["extras"]})
            per.append(entry)
        conv = [p["relres_max_converged"] for p in per if p["relres_max_converged"] is not None]
        eig = {"problems": per, "relres_max_converged": max(conv) if conv else None,
               "with_golden": [p["problem"] for p in per if "golden_ok" in p],
               "golden_ok": all(p.get("golden_ok", True) for p in per),
               "total_s": time.perf_counter() - t0,
               "pipeline": "per problem: Algorithm 1 (q=10) + CholeskyQR2 + projection (mixed) "
                           "+ reduced solve + refinement (FP64 residuals)"}
    bi = sum(v.numel() * 16 for v in Vh)
    bo = sum(b.numel() * 16 for b in Bh)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * step_s, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32+bf16x3", "data": "synthetic",
            "config": {"workload": "batch48", "problems": len(probs_all),
                       "problems_rank0": len(probs),
                       "n_range": [min(m.n for m in meshes), max(m.n for m in meshes)],
                       "entries_per_step": entries, "precision": "mixed",
                       "launch": "grouped persistent kernel in a CUDA graph",
                       "autotuned": info, "autotune_s": tune_s,
                       "parallelism": f"problems sharded by work over {world} ranks",
                       "l2": "flushed between steps (512 MB write)"},
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": entries * args.steps / e2e_total, "unit": UNIT,
                    "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo},
            "gpu_launches": launches, "clocks": clk, "eig_check": eig}
    print(json.dumps(line), flush=True)
    batch.close()
    for c in ctxs:
        c.close()
    return 0


def sustained_bf16_tflops():
    """(peak, source): the sustained dense BF16 rate of MEASURED_PEAKS.json, else the
    profiling recipe's fallback of 1.7 PFLOP/s."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["bf16_tflops_sustained"]), "of measured (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 1700.0, "of fallback (1.7 PFLOP/s sustained)"


def plain_fp64_speedup(bem, ctx, args, prob, mesh, V_res, V_work, B_dev, flush, stream, mixed_rate):
    """The plain FP64 GPU path, for the speedup of the mixed form. Its cost per entry (the
    FP64 evaluation of the 7 points and the 8 nu flops of the contraction) does not depend
    on n; up to n = 20000 it is timed on the workload itself, above that on the workload's
    contour and basis width with the mesh one level coarser cut to 4 nodes (the full FP64
    projection at n = 98304 takes about an hour), beside the mixed path on the same sample."""
    import torch
    c = prob.contour
    n, N, nu = mesh.n, prob.N, prob.nu

    def timed(cx, Vw, Vsrc, prec, B, steps):
        ms = []
        for _ in range(steps):
            flush.fill_(0.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            Vw.copy_(Vsrc, non_blocking=True)
            cx.cholqr2(Vw, want_R=False)
            cx.project(Vw, prec, Bhat=B)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.mean(ms)

    if n <= 20000:
        ms = timed(ctx, V_work, V_res, bem.PREC_FP64, B_dev, args.plain_steps)
        return {"value": n * n * N / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                "steps": args.plain_steps, "speedup_of_mixed": mixed_rate / (n * n * N / (ms * 1e-3)),
                "sample": "the workload itself"}
    import synth
    coarse = {"ellipsoid98304": lambda: synth.tetrakis_sphere(4, (1.0, 0.7, 0.5)),
              "sphere20480": lambda: synth.icosphere(4)}[args.workload]()
    Ns = min(4, N)
    sc = bem.Context(torch.cuda.current_device())
    sc.set_mesh(coarse.xyz, coarse.tri)
    sc.set_contour(c.kind, c.centre, c.a, c.b, Ns)
    Vs = bem.fortran(torch.from_numpy(synth.complex_gaussian(coarse.n, nu, prob.seed)).to(V_res.device))
    Vw = bem.fortran(torch.empty_like(Vs))
    Bs = torch.empty((Ns, nu, nu), dtype=torch.complex128, device=V_res.device)
    timed(sc, Vw, Vs, bem.PREC_FP64, Bs, 1)
    ms64 = timed(sc, Vw, Vs, bem.PREC_FP64, Bs, args.plain_steps)
    timed(sc, Vw, Vs, bem.PREC_MIXED, Bs, 1)
    msmx = timed(sc, Vw, Vs, bem.PREC_MIXED, Bs, max(2, args.plain_steps))
    sc.close()
    ent = float(coarse.n) ** 2 * Ns
    rate64 = ent / (ms64 * 1e-3)
    return {"value": rate64, "unit": UNIT, "ms_per_step": ms64, "steps": args.plain_steps,
            "speedup_of_mixed": mixed_rate / rate64,
            "speedup_of_mixed_same_sample": ms64 / msmx,
            "sample": f"{coarse.name} (n = {coarse.n}), the workload's contour, {Ns} of its "
                      f"{N} nodes, nu = {nu}: FP64 and mixed steps timed on it; "
                      "speedup_of_mixed = the full-size mixed rate over this FP64 rate"}


LARGE_N = 50000   # above this the reported residuals are double-FP32, spot-checked in FP64


def eig_check(ctx, V_res, prec, spec, gold, precision):
    """Solves from V_res and reports every eigenpair inside the contour with its residual
    (FP64; above LARGE_N panels double-FP32, whose entries carry ~1e-13 relative error, and
    the first converged pair recomputed in FP64 beside it), and, with a stored oracle list,
    the per-eigenvalue errors (eig_compare). A failure of the solve is reported in the
    line, not raised."""
    import torch
    import paper_1906_03938_gb300 as bem
    n = V_res.shape[0]
    large = n > LARGE_N
    ctx.set_refine_residual(1 if large else 0)
    t0 = time.perf_counter()
    try:
        lam, X, rel = ctx.solve(V_res, q=10, precision=prec, tol=1e-14)
        torch.cuda.synchronize()
    except Exception as exc:   # the bench line still prints
        ctx.set_refine_residual(0)
        return {"error": str(exc), "solve_s": time.perf_counter() - t0}
    ctx.set_refine_residual(0)
    t_solve = time.perf_counter() - t0
    conv = [k for k in range(len(lam)) if rel[k] <= 1e-8]
    out = {"found": [[l.real, l.imag] for l in lam], "relres": [float(r) for r in rel],
           "converged_inside": len(conv), "relres_max_converged":
               max((float(rel[k]) for k in conv), default=None),
           "solve_s": t_solve, "relres_arith": "double-FP32" if large else "FP64",
           "pipeline": "Algorithm 1 (q=10) + CholeskyQR2 + projection (" + precision +
                       ") + reduced solve + refinement (double-FP32 iterations)"}
    if large and conv:
        k = conv[0]
        r64, _, _ = ctx.residual_arith(np.array([lam[k]]), bem.fortran(X[:, k:k + 1].contiguous()),
                                       arith=0)
        out["fp64_spot_check"] = {"lambda": [lam[k].real, lam[k].imag],
                                  "relres_fp64": float(r64[0]), "relres_double_fp32": float(rel[k])}
    if gold is not None:
        out.update(eig_compare(lam, X.cpu().numpy(), rel, gold, spec, tol=1e-8, conv=1e-8))
    else:
        out["oracle"] = ("no stored oracle eigenvalues for this mesh (the CPU oracle's dense "
                         "FP64 solve is out of reach at this n); each pair is certified by "
                         "its FP64 residual ||A(lambda) x|| / ||x||")
    return out


def run_ours(args):
    import torch
    import paper_1906_03938_gb300 as bem

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prob, mesh, V = problem(args.workload)
    n, N, nu = mesh.n, prob.N, prob.nu
    prec = {"mixed": bem.PREC_MIXED, "fp64": bem.PREC_FP64,
            "hmatrix": bem.PREC_HMATRIX}[args.precision]
    c = prob.contour
    ctx = bem.Context(local)
    ctx.set_twin_clusters(bool(args.twin_clusters))
    stream = torch.cuda.current_stream()
    near_mode = args.near if args.near is not None else (1 if n > 10000 else 0)
    surrogate = None
    if near_mode == 2:
        surrogate = train_surrogate(bem, local)      # untimed: data generation and training
        ctx.surrogate_set(surrogate["params"])
    OPS = {"single": (1.0, 0.0), "neumann": (0.0, 1.0), "robin": (0.5, 1.0)}
    ctx.set_operator(*OPS[args.operator])
    if prec == bem.PREC_HMATRIX:   # low-rank far field: leaves of 32, eta 1, eps 1e-6
        ctx.set_hmatrix(leaf=32, eta=1.0, eps=1e-6, rmax=64)
    if near_mode:
        ctx.set_mesh(mesh.xyz, mesh.tri)
        ctx.set_near_field(near_mode)

    V_host = torch.from_numpy(np.asfortranarray(V)).pin_memory()   # column-major host copy
    V_res = bem.fortran(V_host.to(dev))                              # resident input
    V_work = bem.fortran(torch.empty_like(V_res))
    B_dev = torch.empty((N, nu, nu), dtype=torch.complex128, device=dev)
    B_host = torch.empty((N, nu, nu), dtype=torch.complex128).pin_memory()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    # asynchronous pipeline: the step makes no host synchronisation; the device status of
    # the orthonormalisation is checked after the timed loops
    ctx.set_async(True)

    def step(src):
        ctx.set_mesh(mesh.xyz, mesh.tri)
        ctx.set_contour(c.kind, c.centre, c.a, c.b, N)
        V_work.copy_(src, non_blocking=True)
        ctx.cholqr2(V_work, want_R=False)
        ctx.project(V_work, prec, Bhat=B_dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up
    for _ in range(args.warmup):
        step(V_res)
    barrier()

    # device-resident timing (value) with L2 flushed between steps, per-step events
    ctx.set_timing(True)
    launches0 = ctx.launches
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        step(V_res)
        ev[k][1].record(stream)
    barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    launches = ctx.launches - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    kern_ms = list(ctx.kernel_times())
    ctx.set_timing(False)
    t_total = sum(step_ms) / 1e3

    # end to end through the public API with host buffers: H2D of V and the mesh each
    # step, D2H of the projected matrices
    barrier()
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(float(k))
        e2e_ev[k][0].record(stream)
        step(V_host)
        B_host.copy_(B_dev, non_blocking=True)
        e2e_ev[k][1].record(stream)
    barrier()
    e2e_total = sum(a.elapsed_time(b) for a, b in e2e_ev) / 1e3
    ctx.check()   # device status of every step (raises on a failure)
    # near-field samples of the steps served by the network and by the plain rule
    sur_usage = ctx.surrogate_usage() if near_mode == 2 else None

    # max over ranks
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([t_total, e2e_total], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_total, e2e_total = float(t[0]), float(t[1])

    entries = float(n) * n * N
    value = world * entries * args.steps / t_total
    e2e_value = world * entries * args.steps / e2e_total

    if rank != 0:
        ctx.close()
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0

    # roofline of the dominant kernel
    kern_avg = statistics.mean(kern_ms) if kern_ms else float("nan")
    shape = ctx.mixed_shape()
    if prec == bem.PREC_HMATRIX:
        # low-rank far field: the leaf kernel (dense blocks and the U_b T_b products, one
        # launch per node) dominates. Its algorithmic work is one complex multiply-add per
        # basis column for every dense entry and every rank-1 term of a row: 8 nu flops each,
        # on the FP32 pipe (the entries' own evaluation, 7 points each, goes to the MUFU unit
        # and is not counted). "value" above counts the n^2 N entries of the dense operator
        # that the H-matrix replaces.
        st = ctx.hmatrix_stats()
        work = ctx.hmatrix_work()
        flops = 8.0 * nu * (work["dense_entries"] + work["far_row_terms"])
        peak = ctx.microbench("fp32_fma")
        roof = {"bound": "alu", "pipe": "fp32", "kernel": "hm_leaf_kernel",
                "achieved": flops / (kern_avg * 1e-3) / 1e12, "peak": peak / 1e12,
                "unit": "TFLOP/s", "peak_source": "measured FP32 FMA microbenchmark (bem_microbench)",
                "flops_per_launch": flops, "hmatrix": st, "work_per_node": work,
                "note": "far blocks by adaptive cross approximation (eps 1e-6), dense blocks "
                        "and products in FP32"}
    elif prec == bem.PREC_FP64:
        # plain path: FP64 pipe; algorithmic work = the complex MAC of every entry with
        # every basis column, 8 nu flops per entry
        flops = entries * 8 * nu
        peak = ctx.microbench("fp64_fma")
        roof = {"bound": "alu", "pipe": "fp64", "achieved": flops / (kern_avg * 1e-3) / 1e12,
                "peak": peak / 1e12, "unit": "TFLOP/s",
                "peak_source": "measured FP64 FMA microbenchmark (bem_microbench)"}
    else:
        # mixed path: the MUFU unit binds. Per entry and node the method needs one complex
        # exponential per quadrature point (ex2, sin, cos) and, shared by the G nodes of a
        # unit, one rsqrt per quadrature point. Roof = entries/s if the MUFU unit did only
        # that work at its measured rates.
        rates = {k: ctx.microbench(k) for k in ("ex2", "sin", "cos", "rsqrt")}
        G = unit_nodes(N, nu, 0)
        twins = ctx.node_order()[1]
        clusters = shape["paired"]
        t_entry = mufu_seconds_per_entry(rates, N, G, twins, clusters) / N
        roof = {"bound": "alu", "pipe": "mufu", "achieved": entries / (kern_avg * 1e-3),
                "peak": 1.0 / t_entry, "unit": "entries/s",
                "peak_source": "measured MUFU rates (bem_microbench): "
                               + ", ".join(f"{k} {v:.3e}/s" for k, v in rates.items())
                               + f"; per entry and quadrature point: ex2 per node, sin + cos "
                               f"per node or per twin pair ({twins} of {N // 2} possible), "
                               + (f"rsqrt per twin pair (two-CTA clusters)" if clusters
                                  else f"rsqrt per {G} nodes")}
    if roof.get("peak"):
        roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = measured_traffic(args.workload, args.precision)
    roof["kernel_ms"] = kern_avg if kern_ms else None
    roof["launches_timed"] = len(kern_ms)

    if prec == bem.PREC_MIXED:
        # the tensor pipe: BF16x3 complex contraction, 6 BF16 MMAs of 2 x (2 C) columns per
        # node and 16 K -> 24 nu real flops per entry and node (physical work)
        tflops = 24.0 * nu * entries / (kern_avg * 1e-3) / 1e12
        tpeak, tsrc = sustained_bf16_tflops()
        roof["tensor"] = {"achieved_tflops": tflops, "peak_tflops": tpeak,
                          "frac": tflops / tpeak, "peak_source": "sustained dense BF16 " + tsrc}
        # against the method's own work count (no twin sharing credited) and the smaller of
        # that evaluation bound and the tensor bound (24 nu physical flops per entry and node)
        eval_peak = N / mufu_seconds_method(rates, N)
        tensor_peak = tpeak * 1e12 / (24.0 * nu)
        roof["method_count"] = {
            "eval_peak": eval_peak, "tensor_peak": tensor_peak,
            "frac_eval": roof["achieved"] / eval_peak,
            "frac_min": roof["achieved"] / min(eval_peak, tensor_peak), "unit": "entries/s",
            "peak_source": "per entry and node 7 x (ex2, sin, cos), one rsqrt per quadrature "
                           "point for all N nodes, at the measured MUFU rates; tensor: sustained "
                           "BF16 / (24 nu)"}

    plain = None
    if prec != bem.PREC_FP64 and args.plain_steps > 0:
        plain = plain_fp64_speedup(bem, ctx, args, prob, mesh, V_res, V_work, B_dev, flush,
                                   stream, entries / (t_total / args.steps))

    # accuracy qualifier of the metric (untimed): the eigenpairs inside the contour from
    # this basis (Algorithm 1 basis, CholeskyQR2, projection in the bench's precision,
    # reduced solve, refinement), each with its FP64 residual; against the oracle's discrete
    # eigenvalues where tests/golden stores them
    eig = None
    if not args.no_eig_check and args.operator == "single" and args.precision != "hmatrix":
        eig = eig_check(ctx, V_res, prec, c, read_golden(args.workload + ("_near" if near_mode else "")),
                        args.precision)

    cpu = None
    if not args.no_cpu_baseline and world == 1 and args.operator == "single":
        cpu = oracle_sample(prob, mesh, V)

    bi = V.nbytes + mesh.xyz.nbytes + mesh.tri.nbytes
    bo = N * nu * nu * 16
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {bem.PREC_FP64: "f64", bem.PREC_MIXED: "f32+bf16x3",
                  bem.PREC_HMATRIX: "f32"}[prec], "data": "synthetic",
        "config": {"workload": args.workload, "mesh": mesh.name, "n": n, "N": N, "nu": nu,
                   "contour": f"{c.kind} c={c.centre.real:g} a={c.a:g} b={c.b:g}",
                   "precision": args.precision,
                   "near_field": ["off", "8x8 rule", "surrogate network"][near_mode],
                   "units": shape if prec == bem.PREC_MIXED else None,
                   "operator": args.operator,
                   "parallelism": f"replicas{world}", "l2": "flushed between steps (512 MB write)",
                   "wall_s_timed": wall},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": bi,
                "d2h_bytes_per_step": bo},
        "gpu_launches": launches,
        "clocks": clk,
        "plain_fp64": plain,
        "eig_check": eig,
    }
    if surrogate is not None:
        line["surrogate"] = {k: v for k, v in surrogate.items() if k != "params"}
        net_s, rule_s = sur_usage
        line["surrogate"]["samples_network"] = net_s
        line["surrogate"]["samples_plain_rule"] = rule_s
        line["surrogate"]["network_fraction"] = net_s / max(1, net_s + rule_s)
    print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_inverse_power(args):
    """Algorithm 1 (q steps from a random basis, shift at the contour centre) with the dense
    Schur complement (assembled in FP32, LU-factorised once) and matrix-free (each solve by
    GMRES to relative residual 1e-4 with the fused kernel as the operator); one JSON line with
    both times, the Arnoldi steps, the dense method's n^2 bytes and how far the two bases
    differ in direction."""
    import torch
    import paper_1906_03938_gb300 as bem
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prob, mesh, V = problem(args.workload)
    c = prob.contour
    q = args.inverse_power
    ctx = bem.Context(local)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    ctx.set_contour(c.kind, c.centre, c.a, c.b, prob.N)
    V0 = bem.fortran(torch.from_numpy(V).to(dev))
    out = {}
    for mode in ("dense", "matrix_free"):
        Vw = bem.fortran(V0.clone())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if mode == "dense":
            ctx.inverse_power(Vw, q, c.centre)
            its = 0
        else:
            its = ctx.inverse_power_mf(Vw, q, c.centre, tol=1e-4, max_iter=2000)
        torch.cuda.synchronize()
        out[mode] = (time.perf_counter() - t0, its, Vw)
    Ud, Um = out["dense"][2], out["matrix_free"][2]
    a = (Ud.conj() * Um).sum(0) / (Ud.conj() * Ud).sum(0)
    diff = float(((Um - a[None, :] * Ud).norm(dim=0) / Um.norm(dim=0)).max())
    n = mesh.n
    line = {"metric": "Algorithm 1 inverse power steps", "workload": args.workload, "n": n,
            "N": prob.N, "nu": prob.nu, "q": q,
            "dense_s": out["dense"][0], "matrix_free_s": out["matrix_free"][0],
            "gmres_arnoldi_steps": out["matrix_free"][1], "gmres_tol": 1e-4,
            "dense_S_bytes": n * n * 8, "basis_direction_diff": diff,
            "note": "wall time around each call (synchronised); dense = S assembly + FP32 LU + "
                    "q steps; matrix-free = q steps with GMRES solves, no n^2 storage"}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_sweep_eval_split(args):
    """The fused kernel's time at each split of e^{i phi} between the MUFU sin/cos and the
    FMA-pipe polynomials (bem_set_eval_split 0..4), near field off, mixed precision; the
    measured pipe rates beside it. One JSON line."""
    import torch
    import paper_1906_03938_gb300 as bem
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    prob, mesh, V = problem(args.workload)
    c = prob.contour
    ctx = bem.Context(local)
    ctx.set_mesh(mesh.xyz, mesh.tri)
    ctx.set_contour(c.kind, c.centre, c.a, c.b, prob.N)
    Vd = bem.fortran(torch.from_numpy(V).to(torch.device("cuda", local)))
    B = torch.empty((prob.N, prob.nu, prob.nu), dtype=torch.complex128, device=Vd.device)
    out = {"metric": "fused kernel time by eval split", "workload": args.workload, "n": mesh.n,
           "N": prob.N, "nu": prob.nu, "rates": {k: ctx.microbench(k) for k in (
               "fp32_fma", "fp32x2_fma", "ex2", "sin", "cos", "rsqrt", "sincos_poly")},
           "split": {}}
    for npoly in range(5):
        ctx.set_eval_split(npoly)
        for _ in range(max(1, args.warmup)):
            ctx.project(Vd, bem.PREC_MIXED, Bhat=B)
        torch.cuda.synchronize()
        ctx.set_timing(True)
        for _ in range(args.steps):
            ctx.project(Vd, bem.PREC_MIXED, Bhat=B)
        torch.cuda.synchronize()
        kt = list(ctx.kernel_times())
        ctx.set_timing(False)
        ms = statistics.mean(kt)
        out["split"][npoly] = {"kernel_ms": ms, "entries_per_s": mesh.n ** 2 * prob.N / (ms * 1e-3)}
    ctx.check()
    ctx.close()
    print(json.dumps(out), flush=True)
    return 0


def main():
    args = parse()
    if args.sweep_eval_split:
        return run_sweep_eval_split(args)
    if args.inverse_power > 0:
        return run_inverse_power(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch48":
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
