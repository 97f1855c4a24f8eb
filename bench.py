#!/usr/bin/env python
"""Benchmark of the multi-level power-series solve (arxiv 2307.03968 §IV).

Headline workload (default): S-EFIE PEC sphere of radius 2 wavelengths,
icosphere with 20,480 triangles -> 30,720 RWG unknowns, octree with leaves of
<= 64 unknowns, admissibility dist >= 2 * min(diam), ACA tolerance 1e-4,
complex64 on the GPU, one plane-wave right-hand side (+z incidence, x
polarised).  The operator is built on the GPU (hm_build) and its leaf blocks
factored (hm_factor_leaf) before timing; it stays resident in HBM (about 1.5 GB
of blocks, larger than L2, so no L2 flush is needed between steps).

One step = one hm_powerseries_solve with the paper's settings: leaf level only,
K = 2 terms, plus the FP64-class residual and one refinement step -- the whole
hot path (permute, D^{-1}, K x (near/far product + series accumulate),
residual, correction solve, un-permute).

The default run also measures, in the same process, the other workloads of the
measurement plan under "configs": the 1,920-unknown sphere (latency), the
181-right-hand-side monostatic sweep on the headline operator, the
41,850-unknown dielectric cube with 16 right-hand sides, and a short serving
stream (--no-configs skips them).

Prints ONE JSON line (rank 0).  --impl reference times the CPU oracle instead:
it builds the whole headline operator with the oracle and times series.solve
on it, on one core and on every host core (independent right-hand sides, one
per process).
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

if "--impl" in sys.argv and "reference" in sys.argv:
    # the oracle's solve is numpy on small blocks: one BLAS thread per process, so that
    # "one core" is one core and the all-core run is one process per core
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    # the metric's workload: 30,720 RWG unknowns
    "sphere2": dict(name="sefie_pec_sphere_r2lambda_30720rwg", kind="rwg", subdivisions=5, radius=2.0, leaf_size=64,
                    arity=8, adm=2.0, aca_tol=1e-4, n_terms=2, n_levels=1, refine=True, nrhs=1, unknowns=30720,
                    triangles=20480),
    # the same operator, batched monostatic sweep: 181 RHS (theta 0..180 deg, phi = 0, theta-pol)
    "sphere2_sweep181": dict(name="sefie_pec_sphere_r2lambda_30720rwg_sweep181", kind="rwg", subdivisions=5, radius=2.0,
                             leaf_size=64, arity=8, adm=2.0, aca_tol=1e-4, n_terms=2, n_levels=1, refine=True,
                             nrhs=181, sweep=True, unknowns=30720, triangles=20480),
    # continuous-batching serving stream over a catalog of PEC and dielectric operators
    "serving": dict(name="serving_stream_pec_and_dielectric_catalog", kind="serving", n_requests=2000, seed=5,
                    loads=(0.5, 0.8, 1.0), max_rhs=32, n_slots=4, hbm_budget_gb=64, max_batch_rhs=64,
                    n_terms=2, n_levels=1, refine=True, nrhs=0, unknowns=0),
    # the paper's three experiments (§IV) as synthetic meshes of the stated dimensions, with its settings
    # (binary tree, eq. 7 with eta = 1, ACA 1e-3), one normally incident plane wave, leaf level, K = 2,
    # no refinement (the paper's solve), eps_r = 2 for the dielectrics
    "paper_plate": dict(name="paper_pec_plate_15lambda_67200rwg", kind="rwg", shape=("plate", (15.0, 15.0), (150, 150)),
                        leaf_size=64, arity=2, adm=1.0, aca_tol=1e-3, n_terms=2, n_levels=1, refine=False, nrhs=1,
                        unknowns=67200, triangles=45000),
    "paper_slab": dict(name="paper_dielectric_slab_10x1x0.1lambda_119984swg", kind="swg",
                       shape=("box", (10.0, 1.0, 0.1), (218, 21, 2)), eps=2.0, leaf_size=64, arity=2, adm=1.0,
                       aca_tol=1e-3, n_terms=2, n_levels=1, refine=False, nrhs=1, unknowns=119984, tetrahedra=54936),
    "paper_cylinder": dict(name="paper_hollow_dielectric_cylinder_6lambda_158730swg", kind="swg",
                           shape=("shell", (0.35, 0.4, 6.0), (1, 55, 206)), eps=2.0, leaf_size=64, arity=2, adm=1.0,
                           aca_tol=1e-3, n_terms=2, n_levels=1, refine=False, nrhs=1, unknowns=158730,
                           tetrahedra=67980),
    # the same three at the paper's tree depths (binary levels 6, 10 and 8: leaves of about 1,050, 118 and
    # 621 unknowns), where the paper reports its two-term solve
    "paper_plate_depth6": dict(name="paper_pec_plate_15lambda_67200rwg_depth6", kind="rwg",
                               shape=("plate", (15.0, 15.0), (150, 150)), leaf_size=1050, arity=2, adm=1.0,
                               aca_tol=1e-3, n_terms=2, n_levels=1, refine=False, nrhs=1, unknowns=67200,
                               triangles=45000),
    "paper_slab_depth10": dict(name="paper_dielectric_slab_10x1x0.1lambda_119984swg_depth10", kind="swg",
                               shape=("box", (10.0, 1.0, 0.1), (218, 21, 2)), eps=2.0, leaf_size=118, arity=2,
                               adm=1.0, aca_tol=1e-3, n_terms=2, n_levels=1, refine=False, nrhs=1, unknowns=119984,
                               tetrahedra=54936),
    "paper_cylinder_depth8": dict(name="paper_hollow_dielectric_cylinder_6lambda_158730swg_depth8", kind="swg",
                                  shape=("shell", (0.35, 0.4, 6.0), (1, 55, 206)), eps=2.0, leaf_size=621, arity=2,
                                  adm=1.0, aca_tol=1e-3, n_terms=2, n_levels=1, refine=False, nrhs=1,
                                  unknowns=158730, tetrahedra=67980),
    # the small sphere of the measurement plan (1,920 RWG unknowns, leaf 32): latency, operator L2-resident
    "sphere03": dict(name="sefie_pec_sphere_r0.3lambda_1920rwg", kind="rwg", subdivisions=3, radius=0.3, leaf_size=32,
                     arity=8, adm=2.0, aca_tol=1e-4, n_terms=2, n_levels=1, refine=True, nrhs=1, unknowns=1920,
                     triangles=1280),
    # a smaller sphere of the same family (7,680 unknowns), for profiler captures
    "sphere1": dict(name="sefie_pec_sphere_r1lambda_7680rwg", kind="rwg", subdivisions=4, radius=1.0, leaf_size=64,
                    arity=8, adm=2.0, aca_tol=1e-4, n_terms=2, n_levels=1, refine=True, nrhs=1, unknowns=7680,
                    triangles=5120),
    # V-EFIE: inhomogeneous dielectric cube, side 1 wavelength, 15^3 voxels of 6 tetrahedra
    # (41,850 SWG unknowns), eps_r iid uniform [2, 6], binary tree, eq. 7 with eta = 1, 16 random incidences
    "vefie_cube": dict(name="vefie_dielectric_cube_1lambda_41850swg", kind="swg", voxels=15, side=1.0, eps_lo=2.0,
                       eps_hi=6.0, seed=4, rhs_seed=44, leaf_size=64, arity=2, adm=1.0, aca_tol=1e-4, n_terms=2,
                       n_levels=1, refine=True, nrhs=16, unknowns=41850, tetrahedra=20250),
    # the same element size on a 2/3-wavelength cube (12,600 SWG unknowns), for profiler captures
    "vefie_cube_small": dict(name="vefie_dielectric_cube_0.667lambda_12600swg", kind="swg", voxels=10, side=2.0 / 3.0,
                             eps_lo=2.0, eps_hi=6.0, seed=4, rhs_seed=44, leaf_size=64, arity=2, adm=1.0, aca_tol=1e-4,
                             n_terms=2, n_levels=1, refine=True, nrhs=16, unknowns=12600, tetrahedra=6000),
}
WORKLOAD = WORKLOADS["sphere2"]
METRIC = "power-series solves RHS/s at <=1e-4 rel err vs FP64 oracle; p50/p99 latency"


def workload_mesh(w):
    """(xyz, cells, eps_r or None) of a workload, from the seeded generators."""
    import numpy as np
    import synth
    shape = w.get("shape")
    if shape is not None:
        if shape[0] == "plate":
            xyz, tri = synth.plate(shape[1], shape[2])
            return xyz, tri, None
        xyz, tet = (synth.box_tets(shape[1], shape[2]) if shape[0] == "box" else
                    synth.shell_tets(*shape[1], shape[2]))
        return xyz, tet, np.full(len(tet), w["eps"])
    if w["kind"] == "rwg":
        xyz, tri = synth.icosphere(w["subdivisions"], w["radius"])
        return xyz, tri, None
    xyz, tet = synth.cube_tets(w["voxels"], w["side"])
    return xyz, tet, synth.random_permittivity(len(tet), w["eps_lo"], w["eps_hi"], seed=w["seed"])


def workload_incidences(w):
    import synth
    if w.get("sweep"):
        return synth.monostatic_sweep(w["nrhs"])
    if w.get("shape") is not None:                       # normal incidence on the plate / slab, broadside on the cylinder
        import numpy as np
        return np.array([[0.0, 0.0, -1.0]]) if w["shape"][0] != "shell" else np.array([[1.0, 0.0, 0.0]]), \
            np.array([[1.0, 0.0, 0.0]]) if w["shape"][0] != "shell" else np.array([[0.0, 0.0, 1.0]])
    if w["kind"] == "rwg":
        return synth.plane_wave_z()
    return synth.random_incidences(w["nrhs"], seed=w["rhs_seed"])


def workload_config(w):
    c = {"workload": w["name"], "unknowns": w["unknowns"]}
    if w.get("shape") is not None:
        c.update({"shape": "%s %s, grid %s" % (w["shape"][0], w["shape"][1], w["shape"][2]),
                  "eps_r": w.get("eps"), "tree": "binary (median splits)", "admissibility": "dist>=min(diam) (eta=1)",
                  "rhs": "one plane wave", "leaf_size": w["leaf_size"], "aca_tol": w["aca_tol"],
                  "n_terms": w["n_terms"], "levels": "leaf level only", "refine": "none (the paper's solve)",
                  "nrhs": w["nrhs"], "l2": "operator resident in HBM is larger than L2; no flush",
                  "parallelism": "replicas"})
        return c
    if w["kind"] == "rwg":
        c.update({"triangles": w["triangles"], "radius_lambda": w["radius"], "tree": "octree (median splits)",
                  "admissibility": "dist>=2*min(diam)",
                  "rhs": ("monostatic sweep, theta 0..180 deg step 1, phi 0, theta-pol" if w.get("sweep")
                          else "plane wave +z, x-pol")})
    else:
        c.update({"tetrahedra": w["tetrahedra"], "side_lambda": w["side"],
                  "eps_r": "iid uniform [%g, %g], seed %d" % (w["eps_lo"], w["eps_hi"], w["seed"]),
                  "tree": "binary (median splits)", "admissibility": "dist>=min(diam) (eq. 7, eta=1)",
                  "rhs": "%d plane waves, random incidence and polarisation, seed %d" % (w["nrhs"], w["rhs_seed"])})
    c.update({"leaf_size": w["leaf_size"], "aca_tol": w["aca_tol"], "n_terms": w["n_terms"],
              "levels": "leaf level only", "refine": "one FP64-residual refinement step", "nrhs": w["nrhs"],
              "l2": ("operator resident in HBM is larger than L2; no flush" if w["unknowns"] > 5000 else
                     "operator fits L2 (a latency workload); no flush"), "parallelism": "replicas"})
    return c




def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", default="hm", choices=["hm", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-extras", action="store_true", help="skip the unrefined / full-level / FP64 timings")
    p.add_argument("--no-configs", action="store_true",
                   help="skip the other workloads of the default run (1,920-unknown sphere, 181-RHS sweep, "
                        "dielectric cube, serving stream)")
    p.add_argument("--workload", default="sphere2", choices=sorted(WORKLOADS))
    p.add_argument("--sweep-rhs", type=int, default=None,
                   help="sweep workload: number of monostatic angles (right-hand sides) instead of 181 "
                        "(smaller profiler captures)")
    p.add_argument("--device-loop", action="store_true",
                   help="serving workload: schedule through the device-resident request loop")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU time budget of the oracle sample")
    p.add_argument("--ref-seconds", type=float, default=90.0,
                   help="wall-time budget of the reference arm's timed oracle solves (after its build)")
    p.add_argument("--pin-product", type=int, default=None,
                   help="pin the many-RHS product kernel (0, 8, 16, 32, 1016 = tensor cores) instead of autotuning")
    p.add_argument("--pin-residual", type=int, default=None,
                   help="pin the many-RHS residual kernel (0, 8, 16, 1017 = owner-computes)")
    return p.parse_args()


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return None


PEAKS = _measured_peaks()


def peaks():
    try:
        return float(PEAKS["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------- oracle --------
def oracle_sample_rate(cpu_seconds, warmup=1, steps=None):
    """Time the CPU oracle's power-series solve (series.solve, leaf level, K=2,
    refine) on a sample of the workload's operator: the leaf self blocks of
    S evenly spaced leaves plus every stored near / leaf-level far block whose
    row cluster is one of them.  The time is scaled to the whole operator by
    the ratio of stored complex elements.  Returns a dict for the JSON line."""
    import numpy as np
    from oracle.rwg import RWGMesh
    from oracle.swg import SWGMesh
    from oracle.hmatrix import ClusterTree, HMatrix, partition, recompress
    from oracle import series

    w = WORKLOAD
    xyz, cells, eps = workload_mesh(w)
    mesh = RWGMesh(xyz, cells) if w["kind"] == "rwg" else SWGMesh(xyz, cells, eps)
    tree = ClusterTree(mesh.centres(), *mesh.support_boxes(), w["leaf_size"], w["arity"])
    near_pairs, far_pairs = partition(tree, w["adm"])
    L = tree.depth
    leaves = tree.leaves()
    S = 8
    sample = set(int(i) for i in np.linspace(0, len(leaves) - 1, S).round())
    P = tree.perm
    Hs = HMatrix.__new__(HMatrix)
    Hs.mesh, Hs.tree, Hs.N, Hs.perm, Hs.depth, Hs.n_levels = mesh, tree, tree.N, tree.perm, L, 1
    Hs.leaves = [leaves[i] for i in sorted(sample)]
    Hs.D = []
    for (off, n) in Hs.leaves:
        B = mesh.fill(P[off:off + n], P[off:off + n])
        iu = np.triu_indices(n, 1)
        B[(iu[1], iu[0])] = B[iu]
        Hs.D.append(B)
    Hs.near = []
    for (a, b) in near_pairs:
        if a in sample:
            (io, m), (jo, n) = leaves[a], leaves[b]
            Hs.near.append((io, m, jo, n, mesh.fill(P[io:io + m], P[jo:jo + n])))
    fl = [(a, b) for (a, b) in far_pairs.get(L, []) if a in sample]
    facs = mesh.aca_many([(P[leaves[a][0]:leaves[a][0] + leaves[a][1]], P[leaves[b][0]:leaves[b][0] + leaves[b][1]])
                          for (a, b) in fl], w["aca_tol"])
    Hs.far = {1: []}
    for (a, b), (U, V) in zip(fl, facs):
        U, V = recompress(U, V, w["aca_tol"])
        Hs.far[1].append((leaves[a][0], leaves[a][1], leaves[b][0], leaves[b][1], U, V))
    # element counts of the sample and of the whole leaf-level operator
    samp = sum(n * n for (_, n) in Hs.leaves) + sum(m * n for (_, m, _, n, _) in Hs.near) + \
        sum(U.shape[1] * (m + n) for (_, m, _, n, U, _) in Hs.far[1])
    n_far_total = len(far_pairs.get(L, []))
    mean_far = np.mean([U.shape[1] * (m + n) for (_, m, _, n, U, _) in Hs.far[1]]) if Hs.far[1] else 0.0
    full = sum(n * n for (_, n) in leaves) + sum(leaves[a][1] * leaves[b][1] for (a, b) in near_pairs) + \
        n_far_total * mean_far
    scale = full / samp
    b = mesh.rhs(*workload_incidences(w))
    if b.shape[1] == 1:
        b = b[:, 0]
    for _ in range(warmup):
        series.solve(Hs, b, K=w["n_terms"], levels=1, refine=True)
    times, cpu = [], []
    t_end = time.perf_counter() + cpu_seconds
    n = 0
    while (steps is None and (time.perf_counter() < t_end or n < 3)) or (steps is not None and n < steps):
        c0, t0 = time.process_time(), time.perf_counter()
        series.solve(Hs, b, K=w["n_terms"], levels=1, refine=True)
        times.append(time.perf_counter() - t0)
        cpu.append(time.process_time() - c0)
        n += 1
    t = statistics.median(times) * scale
    cores = max(1, round(sum(cpu) / max(sum(times), 1e-9)))
    nrhs = w["nrhs"]
    return dict(value=nrhs / t, unit="RHS/s", cores=cores, kind="oracle",
                sample="oracle series.solve (K=2, leaf level, refine, %d RHS) on %d of %d leaves with their %d near "
                       "and %d leaf-level far block rows (%.1f%% of the stored elements, far elements of unsampled "
                       "rows estimated from the sample's mean rank); median of %d solves scaled by %.1f; the "
                       "whole-operator oracle, on one core and on all cores, is the --impl reference line"
                       % (nrhs, S, len(leaves), len(Hs.near), len(Hs.far[1]), 100.0 / scale, n, scale),
                solve_s_scaled=t, n_timed=n)


_REF = {}     # the reference arm's oracle operator, inherited by its forked workers


def _ref_worker(reps, ready, go, out):
    """One process of the all-core reference run: `reps` solves of the parent's
    operator (inherited copy-on-write through fork), after the common start."""
    from oracle import series
    w = _REF["w"]
    ready.put(os.getpid())
    go.wait()
    t0 = time.perf_counter()
    for _ in range(reps):
        series.solve(_REF["H"], _REF["b"], K=w["n_terms"], levels=1, refine=w["refine"])
    out.put(time.perf_counter() - t0)


def oracle_reference(w, steps, warmup, budget_s):
    """The reference arm: the oracle builds the WHOLE operator of the workload
    (complex128 fill, ACA, re-compression; the leaf level the solve uses) and
    series.solve is timed on it, unsampled:
      - on one core: `warmup` untimed solves, then single solves until a third
        of the budget is spent (at least one);
      - on every host core: one forked process per core, each solving its own
        copy of the right-hand side `reps` times, all started together; the
        rate is the total number of solves over the wall time.
    No GPU is touched in this process, so forking after the build is safe."""
    import multiprocessing as mp
    import numpy as np
    from oracle.rwg import RWGMesh
    from oracle.swg import SWGMesh
    from oracle.hmatrix import HMatrix
    from oracle import series
    xyz, cells, eps = workload_mesh(w)
    mesh = RWGMesh(xyz, cells) if w["kind"] == "rwg" else SWGMesh(xyz, cells, eps)
    t0 = time.perf_counter()
    H = HMatrix(mesh, leaf_size=w["leaf_size"], arity=w["arity"], adm=w["adm"], aca_tol=w["aca_tol"], levels=1)
    build_s = time.perf_counter() - t0
    b = mesh.rhs(*workload_incidences(w))
    _REF.update(H=H, b=b, w=w)
    for _ in range(warmup):
        series.solve(H, b, K=w["n_terms"], levels=1, refine=w["refine"])
    single, cpu = [], []
    t_end = time.perf_counter() + budget_s / 3.0
    while not single or (time.perf_counter() < t_end and len(single) < max(steps, 1)):
        c0, s0 = time.process_time(), time.perf_counter()
        series.solve(H, b, K=w["n_terms"], levels=1, refine=w["refine"])
        single.append(time.perf_counter() - s0)
        cpu.append(time.process_time() - c0)
    t1 = statistics.median(single)
    P = max(1, os.cpu_count() or 1)
    reps = max(1, min(-(-max(steps, 1) // P), int((budget_s * 2.0 / 3.0) / max(t1, 1e-3) / 2)))
    ctx = mp.get_context("fork")
    ready, out = ctx.Queue(), ctx.Queue()
    go = ctx.Event()
    procs = [ctx.Process(target=_ref_worker, args=(reps, ready, go, out)) for _ in range(P)]
    for p in procs:
        p.start()
    for _ in procs:
        ready.get(timeout=600)
    s0 = time.perf_counter()
    go.set()
    per = [out.get(timeout=3600) for _ in procs]
    wall = time.perf_counter() - s0
    for p in procs:
        p.join(timeout=60)
    n_all = P * reps
    nrhs = b.shape[1]
    st = H.stats()
    return dict(value=n_all * nrhs / wall, steps=n_all, ms_per_step=1e3 * wall / n_all, cores=P, wall_s=wall,
                single_core_value=nrhs / t1, single_core_ms=1e3 * t1, single_core_steps=len(single),
                single_core_cores_used=max(1, round(sum(cpu) / max(sum(single), 1e-9))), build_s=build_s,
                worker_s=[round(v, 3) for v in per],
                sample="the whole leaf-level operator built by the oracle (%d unknowns, %d near blocks with %d "
                       "elements, %d leaf-level far blocks with %d elements, %d leaf self blocks; build %.0f s on "
                       "%d cores); series.solve (K=%d, leaf level, refine=%s, %d RHS) timed %d times on one core "
                       "(median %.2f s) and %d times on %d cores (%d processes x %d solves, all started together, "
                       "%.2f s wall)"
                       % (H.N, st["near_blocks"], st["near_elems"], st["far_blocks"].get(1, 0),
                          st["far_elems"].get(1, 0), st["leaves"], build_s, P, w["n_terms"], w["refine"], nrhs,
                          len(single), t1, n_all, P, P, reps, wall))


# ---------------------------------------------------------------- clocks --------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(gpu)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- traffic -------
def committed_traffic():
    """Per-launch DRAM traffic of the product kernel from the committed ncu
    summary, if it was taken on the current kernel source (k_product.cu and the
    headers holding its device code); else None."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    csrc = os.path.join(ROOT, "paper_2307_03968_gb300", "csrc")
    try:
        with open(path) as f:
            d = json.load(f)
        h = hashlib.sha256(b"".join(open(os.path.join(csrc, f), "rb").read()
                                    for f in ("k_product.cu", "k_product_dev.cuh", "k_common.cuh"))).hexdigest()[:16]
        if d.get("k_product_sha256_16") == h and d.get("workload") == WORKLOAD["name"]:
            return d.get("bytes_per_launch")
    except Exception:
        pass
    return None


# ---------------------------------------------------------------- ranks ---------
def max_over_ranks(ms, dist, device):
    """The slowest rank's time (every rank gets it): the timed region of a job
    ends when its last replica ends."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(steps, nrhs, world, ms):
    """Whole-job right-hand sides per second: every rank is an independent replica
    solving `steps` x `nrhs` right-hand sides in (at most) `ms` milliseconds."""
    return steps * nrhs * world / (ms / 1e3)


# ---------------------------------------------------------------- timing --------
def timed_solves(A, b, x, opts, K, W, stream, barrier, local):
    """W untimed solves, then K solves each bracketed by CUDA events on the launching
    stream, with nvidia-smi clocks sampled over the timed region.  Returns (total
    ms from the first start to the last end, sorted per-solve ms, clocks)."""
    import torch
    for _ in range(W):
        A.solve(b, x, **opts)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    clocks = ClockSampler(local)
    time.sleep(0.3)
    barrier()
    for i in range(K):
        starts[i].record(stream)
        A.solve(b, x, **opts)
        ends[i].record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    total_ms = starts[0].elapsed_time(ends[-1])
    lat = sorted(s.elapsed_time(e) for s, e in zip(starts, ends))
    return total_ms, lat, clk


def pct(lat, q):
    return lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))]


def product_roofline(A, b, x, opts, nrhs, Kp, sm_max):
    """The same solves launched kernel by kernel, with CUDA events around every
    launch of the block-product kernel on its stream (graph replay hides them);
    achieved = algorithmic bytes (or flops) per launch / mean launch time.
    Returns (roofline dict, eager ms per solve)."""
    import torch
    stream = torch.cuda.current_stream()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    A.profile(True)
    p0.record(stream)
    for _ in range(Kp):
        A.solve(b, x, graph=False, **opts)
    p1.record(stream)
    torch.cuda.synchronize()
    prof_ms, prof_n, prof_bytes = A.profile_read()
    A.profile(False)
    eager_ms = p0.elapsed_time(p1) / Kp
    peak, peak_kind = peaks()
    per_launch_bytes = prof_bytes / max(prof_n, 1)
    per_launch_ms = prof_ms / max(prof_n, 1)
    # every stored complex element is used twice per right-hand side (the block and its
    # half-storage mirror): 2 complex multiply-adds = 16 real flops per 8 bytes per RHS
    flops_per_launch = 2.0 * per_launch_bytes * nrhs
    alu_peak = 152 * 128 * 2 * (sm_max or 2070.0) * 1e6 / 1e12      # FP32 FMA lanes x 2 flops x clock (TFLOP/s)
    prod_choice = A.tuning(nrhs)[0] if nrhs >= 4 else 0
    if prod_choice == 1016:
        # tensor-core product (3xTF32): three TF32 MMAs per useful FP32-accurate product, so its roof is
        # the TF32 tensor peak / 3; the TF32 peak is the measured sustained bf16 peak x the nominal
        # TF32/bf16 ratio (1.1 / 2.25 PFLOP/s dense)
        bf16_s = (PEAKS or {}).get("bf16_tflops_sustained")
        tf32 = (bf16_s if bf16_s else 1700.0) * 1.1 / 2.25
        bound, unit, rpeak = "tensor", "TFLOP/s", tf32 / 3.0
        rkind = ("measured sustained bf16 %.1f TFLOP/s x 1.1/2.25 (TF32) / 3 (3xTF32 products)" % bf16_s
                 if bf16_s else "fallback 1.7 PFLOP/s bf16 sustained x 1.1/2.25 / 3")
        kernel = ("k_split_x + k_tc_stage1 (low-rank stage 1 batched over shared input clusters) + k_apply_tc "
                  "(dense products and second stages; tcgen05 kind::tf32, 3xTF32; units of <= 64 K chunks; blocks "
                  "<= 64 x 64, rank <= 32) + k_apply_items for larger blocks (k_mrhs_tc.cu, k_product.cu)")
    elif flops_per_launch / (alu_peak * 1e12) > per_launch_bytes / (peak * 1e9):
        bound, unit, rpeak = "alu", "TFLOP/s", alu_peak
        rkind = "derived: 152 SMs x 128 FP32 lanes x 2 flops x max SM clock"
        kernel = ("k_apply_mrhs<%d> (shared-memory SIMT, %d RHS per chunk) + k_apply_items for larger blocks "
                  "(k_mrhs.cu, k_product.cu)" % (prod_choice, prod_choice) if prod_choice
                  else "k_apply_items<float,float,3> (one RHS at a time, k_product.cu)")
    else:
        bound, unit, rpeak, rkind = "hbm", "GB/s", peak, peak_kind
        kernel = "k_apply_items<float,float,3> (near + leaf-level far block product, k_product.cu)"
    achieved = None
    if prof_n:
        achieved = (flops_per_launch / (per_launch_ms * 1e-3) / 1e12 if unit == "TFLOP/s"
                    else per_launch_bytes / (per_launch_ms * 1e-3) / 1e9)
    roof = {"bound": bound, "kernel": kernel, "achieved": achieved, "peak": rpeak, "peak_kind": rkind, "unit": unit,
            "frac": (achieved / rpeak) if achieved else None, "traffic": None,
            "bytes_per_launch": per_launch_bytes, "flops_per_launch": flops_per_launch, "nrhs": nrhs,
            "ms_per_launch": per_launch_ms, "launches": prof_n,
            "hbm_gbs": per_launch_bytes / (per_launch_ms * 1e-3) / 1e9 if prof_n else None,
            "share_of_step": (prof_ms / Kp / eager_ms) if eager_ms else None,
            "measured_on": "the timed solve launched kernel by kernel (%d steps, %.4f ms/step)" % (Kp, eager_ms)}
    return roof, eager_ms


def series_report(A, si):
    """Convergence of the series on this operator (the library's estimates of
    ||D^-1 M_l||_2 and of the spectral radius per level, hm_estimate_norms) and the
    relative residual |b - A x| / |b| of the refined solution (max over columns)."""
    info = A.info()
    nl = max(1, min(info.n_levels, 16))
    return {"rel_residual": si.rel_residual, "convergent": si.convergent, "norm_iters": info.norm_iters,
            "norm_est": [round(v, 6) for v in info.norm_est[:nl]],
            "rho_est": [round(v, 6) for v in info.rho_est[:nl]],
            "note": "norm_est / rho_est per level (level 1 = leaf); the K-term series converges to A^-1 b "
                    "only where rho < 1; parity is against the oracle running the same K-term algorithm"}


def one_launch_timing(A, b, x, opts, K, W, stream, barrier, local):
    """The same solve as ONE cooperative kernel (hm_solve_opts.persistent, graph
    replayed): per-solve latency and rate, and its largest difference from the
    multi-kernel solve's result."""
    import numpy as np
    import torch
    ref = x.clone()
    A.solve(b, ref, **opts)
    si = A.solve(b, x, info=True, persistent=True, **opts)
    torch.cuda.synchronize()
    r, g = ref.cpu().numpy(), x.cpu().numpy()
    diff = float(max(np.linalg.norm(g[j] - r[j]) / np.linalg.norm(r[j]) for j in range(r.shape[0])))
    total, lat, clk = timed_solves(A, b, x, dict(opts, persistent=True), K, W, stream, barrier, local)
    return {"value": K * b.shape[0] / (total / 1e3), "unit": "RHS/s", "ms_per_step": total / K,
            "p50_ms": pct(lat, 0.5), "p99_ms": pct(lat, 0.99), "kernel_launches": int(si.kernel_launches),
            "max_rel_diff_vs_multi_kernel": diff, "clocks": clk}


def gpu_build(w):
    from paper_2307_03968_gb300.hm import HMatrix
    xyz, cells, eps = workload_mesh(w)
    t0 = time.perf_counter()
    A = HMatrix.build(xyz, cells, eps_r=eps, leaf_size=w["leaf_size"], arity=w["arity"], adm=w["adm"],
                      aca_tol=w["aca_tol"], levels=-1)
    A.factor_leaf()
    return A, time.perf_counter() - t0


def config_line(w, A, nrhs, total_ms, K, lat, clk, roof, si, build_s, tuning=None, note=None):
    c = workload_config(w)
    c["nrhs"] = nrhs
    d = {"config": c, "value": K * nrhs / (total_ms / 1e3), "unit": "RHS/s", "steps": K,
         "ms_per_step": total_ms / K, "p50_ms": pct(lat, 0.5), "p99_ms": pct(lat, 0.99), "build_s": build_s,
         "roofline": roof, "series": series_report(A, si), "clocks": clk}
    if tuning is not None:
        d["tuning"] = dict(zip(("product_kernel", "residual_kernel", "product_ms", "residual_ms"), tuning))
    if note:
        d["note"] = note
    return d


def extra_configs(A2, local, barrier):
    """The other workloads of the measurement plan, timed in the same process as
    the headline (graph-replayed solves, CUDA events on the launching stream)."""
    import torch
    stream = torch.cuda.current_stream()
    out = {}
    # config 1: 1,920-unknown sphere, 1 RHS: latency of single solves (operator L2-resident)
    w = WORKLOADS["sphere03"]
    A, bs = gpu_build(w)
    b = torch.empty((1, A.n), dtype=torch.complex64, device="cuda")
    A.rhs_plane_wave(*workload_incidences(w), b)
    x = torch.empty_like(b)
    opts = dict(n_terms=w["n_terms"], n_levels=w["n_levels"], refine=w["refine"])
    si = A.solve(b, x, info=True, **opts)
    total, lat, clk = timed_solves(A, b, x, opts, 300, 20, stream, barrier, local)
    out["sphere03"] = config_line(w, A, 1, total, 300, lat, clk, None, si, bs,
                                  note="operator %.1f MB, L2-resident: latency, no roofline line"
                                       % (A.info().device_bytes / 1e6))
    out["sphere03"]["launches_per_step"] = int(si.kernel_launches)
    out["sphere03"]["one_launch"] = one_launch_timing(A, b, x, opts, 300, 20, stream, barrier, local)
    A.close()
    # config 3: the headline operator, 181-RHS monostatic sweep (autotuned kernels)
    w = WORKLOADS["sphere2_sweep181"]
    kh, ph = workload_incidences(w)
    b = torch.empty((len(kh), A2.n), dtype=torch.complex64, device="cuda")
    A2.rhs_plane_wave(kh, ph, b)
    x = torch.empty_like(b)
    opts = dict(n_terms=w["n_terms"], n_levels=w["n_levels"], refine=w["refine"])
    si = A2.solve(b, x, info=True, **opts)                 # autotunes the 256-RHS bucket, then solves
    total, lat, clk = timed_solves(A2, b, x, opts, 6, 2, stream, barrier, local)
    roof, _ = product_roofline(A2, b, x, opts, len(kh), 2, (clk or {}).get("sm_max_mhz"))
    out["sphere2_sweep181"] = config_line(w, A2, len(kh), total, 6, lat, clk, roof, si, 0.0,
                                          tuning=A2.tuning(len(kh)),
                                          note="the headline operator (built once)")
    del b, x
    # config 4: dielectric cube, 41,850 SWG unknowns, 16 RHS
    w = WORKLOADS["vefie_cube"]
    A, bs = gpu_build(w)
    kh, ph = workload_incidences(w)
    b = torch.empty((len(kh), A.n), dtype=torch.complex64, device="cuda")
    A.rhs_plane_wave(kh, ph, b)
    x = torch.empty_like(b)
    opts = dict(n_terms=w["n_terms"], n_levels=w["n_levels"], refine=w["refine"])
    si = A.solve(b, x, info=True, **opts)
    total, lat, clk = timed_solves(A, b, x, opts, 10, 3, stream, barrier, local)
    roof, _ = product_roofline(A, b, x, opts, len(kh), 3, (clk or {}).get("sm_max_mhz"))
    out["vefie_cube"] = config_line(w, A, len(kh), total, 10, lat, clk, roof, si, bs, tuning=A.tuning(len(kh)))
    A.close()
    del b, x
    torch.cuda.synchronize()
    # config 5: a short serving stream (cold start, saturation, Poisson arrivals at 0.5, 0.8 and 1.0 of it)
    out["serving"] = serving_run(WORKLOADS["serving"], n_requests=300, loads=(0.5, 0.8, 1.0), sat_requests=200,
                                 local=local)
    out["serving_device_loop"] = serving_run(WORKLOADS["serving"], n_requests=300, loads=(0.5, 0.8, 1.0),
                                             sat_requests=200, local=local, device_loop=True)
    return out


# ---------------------------------------------------------------- main ----------
def main():
    a = parse()
    global WORKLOAD
    WORKLOAD = WORKLOADS[a.workload]
    if a.sweep_rhs and WORKLOAD.get("sweep"):
        WORKLOAD = dict(WORKLOAD, nrhs=a.sweep_rhs, name=WORKLOAD["name"].replace("181", str(a.sweep_rhs)))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    w = WORKLOAD
    if w["kind"] == "serving":
        if a.impl == "reference":
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable": "the oracle has no serving path; "
                                  "its solve rate is the --impl reference line of the other workloads"}))
            return
        if rank == 0:
            import torch
            torch.cuda.set_device(local)
            serving_main(a, w)
        return
    config = workload_config(w)

    if a.impl == "reference":
        if rank != 0:
            return
        warm = min(a.warmup, 1)
        r = oracle_reference(w, a.steps, warm, a.ref_seconds)
        line = {"impl": "reference", "metric": METRIC, "value": r["value"], "unit": "RHS/s", "n_gpus": a.gpus,
                "steps": r["steps"], "warmup": warm, "ms_per_step": r["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
                "data": "synthetic", "config": config,
                "cpu_baseline": {"value": r["value"], "unit": "RHS/s", "cores": r["cores"], "kind": "oracle",
                                 "sample": r["sample"], "single_core_value": r["single_core_value"],
                                 "single_core_ms": r["single_core_ms"], "single_core_steps": r["single_core_steps"],
                                 "oracle_build_s": r["build_s"], "all_core_wall_s": r["wall_s"]},
                "e2e": {"value": r["value"], "unit": "RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_2307_03968_gb300.hm import HMatrix
    xyz, cells, eps = workload_mesh(w)
    t0 = time.perf_counter()
    want_fp64 = not a.no_extras and w["nrhs"] == 1          # for the plain FP64 single-solve comparator
    A = HMatrix.build(xyz, cells, eps_r=eps, leaf_size=w["leaf_size"], arity=w["arity"], adm=w["adm"],
                      aca_tol=w["aca_tol"], levels=-1, keep_fp64=want_fp64)
    build_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    A.factor_leaf()
    factor_s = time.perf_counter() - t0
    info = A.info()
    kh, ph = workload_incidences(w)
    nrhs = len(kh)
    b = torch.empty((nrhs, A.n), dtype=torch.complex64, device="cuda")
    A.rhs_plane_wave(kh, ph, b)
    x = torch.empty_like(b)
    opts = dict(n_terms=w["n_terms"], n_levels=w["n_levels"], refine=w["refine"])
    if nrhs >= 4 and (a.pin_product is not None or a.pin_residual is not None):
        A.set_tuning(nrhs, a.pin_product if a.pin_product is not None else 16,
                     a.pin_residual if a.pin_residual is not None else 8)
    si = A.solve(b, x, info=True, **opts)
    launches_per_step = si.kernel_launches
    stream = torch.cuda.current_stream()
    K = a.steps
    total_ms, lat, clk = timed_solves(A, b, x, opts, K, a.warmup, stream, barrier, local)
    roof, eager_ms = product_roofline(A, b, x, opts, nrhs, min(K, 1000), (clk or {}).get("sm_max_mhz"))
    if roof["bound"] == "hbm":
        roof["traffic"] = committed_traffic()
    total_ms = max_over_ranks(total_ms, dist, "cuda")
    value = replica_rate(K, nrhs, world, total_ms)

    # extras: unrefined solve and full-level solve (nested, all levels)
    def time_plain(n, **kw):
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(3):
            A.solve(b, x, **kw)
        s0.record(stream)
        for _ in range(n):
            A.solve(b, x, **kw)
        s1.record(stream)
        torch.cuda.synchronize()
        return s0.elapsed_time(s1) / n
    no_refine_ms = full_nested_ms = full_flat_ms = fp64_ms = None
    if want_fp64:
        # the plain FP64 path: complex128 blocks and vectors, one right-hand side per call (no refinement:
        # it is already FP64)
        b64 = b.to(torch.complex128)
        x64 = torch.empty_like(b64)
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(3):
            A.solve(b64, x64, n_terms=w["n_terms"], n_levels=w["n_levels"], fp64=True)
        s0.record(stream)
        for _ in range(20):
            A.solve(b64, x64, n_terms=w["n_terms"], n_levels=w["n_levels"], fp64=True)
        s1.record(stream)
        torch.cuda.synchronize()
        fp64_ms = s0.elapsed_time(s1) / 20
        del b64, x64
    if not a.no_extras:
        no_refine_ms = time_plain(200, n_terms=2, n_levels=1, refine=False)
        # the nested form costs ~(K+1)^levels leaf-level products: few repetitions on deep trees, none past 6
        if info.n_levels <= 6:
            full_nested_ms = time_plain(20 if info.n_levels <= 3 else 2, n_terms=2, n_levels=-1, nested=True,
                                        refine=False)
        full_flat_ms = time_plain(100, n_terms=2, n_levels=-1, nested=False, refine=False)

    # the same solve as one cooperative kernel (the multi-kernel graph replay is the headline)
    one_launch = None
    if not a.no_extras and nrhs == 1:
        one_launch = one_launch_timing(A, b, x, opts, min(K, 200), 5, stream, barrier, local)

    # end to end through the host-buffer entry point
    e2e = None
    if not a.no_e2e:
        # page-locked host buffers (the library copies them directly)
        bh = b.cpu().pin_memory().numpy()
        xh = torch.empty(b.shape, dtype=b.dtype).pin_memory().numpy()
        for _ in range(3):
            A.solve_host(bh, out=xh, **opts)
        Ke = max(10, min(K, 500))
        barrier()
        t0 = time.perf_counter()
        for _ in range(Ke):
            A.solve_host(bh, out=xh, **opts)
            _ = float(np.abs(xh[0, 0]))
        dt = time.perf_counter() - t0
        e2e = {"value": Ke * nrhs * world / dt, "unit": "RHS/s", "h2d_bytes_per_step": int(bh.nbytes),
               "d2h_bytes_per_step": int(xh.nbytes), "steps": Ke}

    configs = None
    if rank == 0 and world == 1 and a.workload == "sphere2" and not a.no_configs:
        configs = extra_configs(A, local, barrier)

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        try:
            r = oracle_sample_rate(a.cpu_seconds)
            cpu = {k: r[k] for k in ("value", "unit", "cores", "kind", "sample")}
        except Exception as ex:  # the baseline is reported, never required
            cpu = {"value": None, "unit": "RHS/s", "cores": None, "kind": "oracle", "sample": "failed: %r" % ex}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": world, "steps": K, "warmup": a.warmup,
                "ms_per_step": total_ms / K, "p50_ms": pct(lat, 0.5), "p99_ms": pct(lat, 0.99),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64",
                "data": "synthetic", "config": config, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clk, "gpu_launches": int(launches_per_step) * K, "series": series_report(A, si),
                "configs": configs,
                "extras": {"eager_ms_per_step": eager_ms, "build_s": build_s, "factor_s": factor_s,
                           "no_refine_ms": no_refine_ms, "fp64_plain_ms": fp64_ms,
                           "fp64_plain_rhs_s": (1e3 / fp64_ms) if fp64_ms else None,
                           "full_level_nested_ms": full_nested_ms, "full_level_flat_ms": full_flat_ms,
                           "one_launch": one_launch,
                           "n_levels": info.n_levels, "near_blocks": info.n_near,
                           "far_blocks": [info.n_far[i] for i in range(info.n_levels)],
                           "max_rank": info.max_rank, "device_bytes": info.device_bytes,
                           "tuning": (dict(zip(("product_rhs_chunk", "residual_rhs_chunk", "product_ms",
                                                "residual_ms"), A.tuning(nrhs))) if nrhs >= 4 else None),
                           "launches_per_step": int(launches_per_step)}}
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------- serving -------
def serving_catalog(seed, full=False):
    """Seeded catalog of scatterers, meshed at about a tenth of a wavelength (PEC
    surfaces, RWG) or a fifteenth (dielectric volumes, SWG).  Returns a list of
    dicts (name, xyz, cells, eps_r or None, tree options).

    full=False: 12 operators (3 spheres, 3 cubes, 3 closed cylinders, 3
    dielectric cubes of 6,528-21,600 unknowns), built in seconds.  full=True:
    the 24 of the serving workload's description: 18 PEC bodies (6 spheres of
    radius 0.7-3.2 wavelengths, 6 cubes and 6 closed cylinders of 0.5-3
    wavelengths; 882 to 30,720 RWG unknowns: meshed at a tenth of a wavelength,
    bodies of this size have no more) and 6 inhomogeneous dielectric cubes of
    6,528 to 41,850 SWG unknowns (eps_r uniform [2, 6])."""
    import numpy as np
    import synth
    rng = np.random.default_rng(seed)
    rwg = dict(leaf_size=64, arity=8, adm=2.0)
    swg = dict(leaf_size=64, arity=2, adm=1.0)
    k = 2 if full else 1
    cat = []
    for s_ in (3, 4, 5) * k:                                # spheres: edge ~ radius / (1.1 * 2^s)
        r = 1.1 * 2 ** s_ / 10.0 * rng.uniform(0.8, 1.0)
        xyz, tri = synth.icosphere(s_, r)
        cat.append(dict(name="pec_sphere_r%.2f" % r, xyz=xyz, cells=tri, eps_r=None, opts=rwg))
    for _ in range(3 * k):                                  # cubes
        a = rng.uniform(0.5, 3.0)
        n = int(np.ceil(10 * a))
        xyz, tri = synth.box_surface((a, a, a), (n, n, n))
        cat.append(dict(name="pec_cube_a%.2f" % a, xyz=xyz, cells=tri, eps_r=None, opts=rwg))
    for _ in range(3 * k):                                  # closed cylinders
        r, h = rng.uniform(0.25, 1.0 if not full else 1.5), rng.uniform(0.5, 3.0)
        xyz, tri = synth.closed_cylinder(r, h, int(np.ceil(2 * np.pi * r * 10)), int(np.ceil(10 * h)),
                                         int(np.ceil(10 * r)))
        cat.append(dict(name="pec_cylinder_r%.2f_h%.2f" % (r, h), xyz=xyz, cells=tri, eps_r=None, opts=rwg))
    for n in ((8, 10, 11, 12, 13, 15) if full else (8, 10, 12)):   # dielectric cubes, side n / 15
        xyz, tet = synth.cube_tets(n, n / 15.0)
        eps = synth.random_permittivity(len(tet), 2.0, 6.0, seed=seed + n)
        cat.append(dict(name="dielectric_cube_%dvox" % n, xyz=xyz, cells=tet, eps_r=eps, opts=swg))
    return cat


def serving_run(w, n_requests, loads, sat_requests, local=0, device_loop=False, full=False):
    """Serving stream (config-5 shape) through the continuous-batching server
    (hm_server_*, the library's public serving API): requests of 1..max_rhs
    right-hand sides on operators drawn uniformly from the catalog, host buffers
    in and out.  Phases: cold start (one request per operator: build + factor +
    first solve), saturation (sat_requests queued at once), then Poisson arrivals
    at the given fractions of the saturation throughput, n_requests each.
    Latency = submit to completion as measured by the server.  Returns a dict."""
    import threading
    import numpy as np
    from paper_2307_03968_gb300.hm import Server
    rng = np.random.default_rng(w["seed"])
    cat = serving_catalog(w["seed"], full=full)
    srv = Server(n_slots=w["n_slots"], hbm_budget_bytes=int(w["hbm_budget_gb"] * 2 ** 30),
                 max_batch_rhs=w["max_batch_rhs"], device_loop=device_loop)
    ops = []
    for g in cat:
        op, n = srv.add_mesh(g["xyz"], g["cells"], eps_r=g["eps_r"], aca_tol=1e-4, levels=-1, n_terms=w["n_terms"],
                             n_levels=w["n_levels"], nested=True, refine=w["refine"], **g["opts"])
        pool = (rng.normal(size=(w["max_rhs"], n)) + 1j * rng.normal(size=(w["max_rhs"], n))).astype(np.complex64)
        ops.append(dict(op=op, n=n, name=g["name"], pool=pool))
    # cold start: one request per operator, sequentially
    cold = []
    for o in ops:
        x, lat = srv.wait(srv.submit(o["op"], o["pool"][:8]))
        cold.append(lat)

    def draw(k):
        return [(int(rng.integers(len(ops))), int(rng.integers(1, w["max_rhs"] + 1))) for _ in range(k)]

    def run(reqs, rate=None):
        """Submit (op, R) requests (all at once if rate is None, else Poisson at
        `rate` requests/s); returns (rhs/s, latencies ms, wall s)."""
        lats = [None] * len(reqs)
        ids = [None] * len(reqs)
        ready = threading.Semaphore(0)

        def waiter():
            for i in range(len(reqs)):
                ready.acquire()
                lats[i] = srv.wait(ids[i])[1]
        th = threading.Thread(target=waiter)
        th.start()
        gaps = rng.exponential(1.0 / rate, len(reqs)) if rate else np.zeros(len(reqs))
        t0 = time.perf_counter()
        t_next = t0
        for i, (k, r) in enumerate(reqs):
            t_next += gaps[i]
            dt = t_next - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            ids[i] = srv.submit(ops[k]["op"], ops[k]["pool"][:r])
            ready.release()
        th.join()
        wall = time.perf_counter() - t0
        return sum(r for _, r in reqs) / wall, lats, wall

    n_req = n_requests
    clocks = ClockSampler(local)
    sat, _, _ = run(draw(sat_requests))
    mean_r = (w["max_rhs"] + 1) / 2.0
    res = []
    for f in loads:
        reqs = draw(n_req)
        thr, lats, wall = run(reqs, rate=f * sat / mean_r)
        lats = np.sort(np.array(lats))
        res.append({"offered": f, "offered_rhs_s": f * sat, "achieved_rhs_s": thr, "requests": len(reqs),
                      "p50_ms": float(np.percentile(lats, 50)), "p99_ms": float(np.percentile(lats, 99)),
                      "wall_s": wall})
    info = srv.info()
    srv.close()
    clk = clocks.stop()
    mid = min(res, key=lambda d: abs(d["offered"] - 0.8))
    return {"config": {"workload": w["name"], "operators": [dict(name=o["name"], unknowns=o["n"]) for o in ops],
                       "requests_per_load": n_req, "saturation_requests": sat_requests,
                       "rhs_per_request": "uniform 1..%d" % w["max_rhs"], "arrivals": "Poisson, seed %d" % w["seed"],
                       "solve": "leaf level, K=2, one refinement", "slots": w["n_slots"],
                       "hbm_budget_gb": w["hbm_budget_gb"], "max_batch_rhs": w["max_batch_rhs"]},
            "value": mid["achieved_rhs_s"], "unit": "RHS/s", "p50_ms": mid["p50_ms"], "p99_ms": mid["p99_ms"],
            "saturation_rhs_s": sat, "loads": res,
            "cold_ms": {"p50": float(np.percentile(cold, 50)), "max": float(np.max(cold))},
            "batches": info.batches, "solved_rhs": info.solved_rhs, "builds": info.builds,
            "evictions": info.evictions, "peak_resident_gb": info.peak_resident_bytes / 2 ** 30, "clocks": clk,
            "scheduler": ("device-resident request loop (one cooperative kernel serving a ring; %d launches, "
                          "%d stops for builds and recordings)" % (info.loop_launches, info.loop_stops)
                          if device_loop else "host thread launching graph-replayed solves on %d streams"
                          % w["n_slots"]),
            "note": "every request is end to end: host b in, host x out; value = achieved RHS/s at the load "
                    "nearest 0.8 of saturation"}


def serving_main(a, w):
    """The serving workload as the headline line (bench.py --workload serving)."""
    s = serving_run(w, w["n_requests"], w["loads"], max(200, w["n_requests"] // 4), device_loop=a.device_loop,
                    full=True)
    main = s["loads"][-1]
    line = {"metric": METRIC, "value": main["achieved_rhs_s"], "unit": "RHS/s", "n_gpus": 1,
            "steps": sum(d["requests"] for d in s["loads"]), "warmup": len(s["config"]["operators"]),
            "ms_per_step": None, "p50_ms": s["p50_ms"], "p99_ms": s["p99_ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": dict(s["config"], parallelism="replicas"), "roofline": None, "cpu_baseline": None,
            "e2e": {"value": main["achieved_rhs_s"], "unit": "RHS/s", "h2d_bytes_per_step": None,
                    "d2h_bytes_per_step": None,
                    "note": "every serving request is end to end: host b in, host x out"},
            "clocks": s["clocks"],
            "serving": {k: s[k] for k in ("saturation_rhs_s", "loads", "cold_ms", "batches", "solved_rhs", "builds",
                                          "evictions", "peak_resident_gb", "scheduler")}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
