#!/usr/bin/env python
"""Benchmark of the phase-field fracture hot path on one GB300 (or N replicas).

Default workload: the 2D notched specimen with Q2 elements on 256 x 256 cells (789,507 DoFs),
seeded state u ~ N(0, (1e-3)^2), phi ~ U(0.9, 1) with phi = 0 on the slit, phi_old slightly above
phi (about half of the phase-field DoFs end up in the active set). One step is one pass of the
whole hot path: set_state with the active set of Alg. 1, then one Newton step: residual, active
set, residual of the projected state, per-point tangent data, multigrid setup (state transfer,
diagonals, eigenvalue estimates, dense coarse inverses), flexible GMRES with the monolithic GMG
preconditioner to 1e-6, and the Newton update. The multigrid runs in FP32 (mixed precision)
unless --mg-precision 64; the outer FP64 operator in double-word arithmetic unless --fp64-mode 0.

value = DoFs processed per second of full Newton steps (n_dofs * steps / time, summed over
ranks). Extra keys: the Jacobian-apply sweep (p = 1..4, FP64 and FP32), the Newton step with the
FP64 multigrid, the full active-set solve to the 1e-8 Newton tolerance with the mixed and with the
plain FP64 multigrid (pdas_1e8; its final residual recomputed by the oracle), the error of the
Newton update against the oracle's direct-solve step (oracle_error), the roofline of the dominant
kernel, the end-to-end figure through host buffers (the mean over the same number of steps as
value), SM clocks during the timed region and the CPU oracle baseline. The oracle runs only in the
CPU leg (rank 0 at N = 1; --no-cpu skips it), after the GPU timings.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
METRIC = "Jacobian-apply DoF/s (% HBM roofline) and s per Newton step, FP64 vs mixed GMG"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12  # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--dim", type=int, default=2)
    ap.add_argument("--degree", type=int, default=2)
    ap.add_argument("--cells", type=int, default=256)
    ap.add_argument("--split", type=int, default=1)
    ap.add_argument("--mg-precision", type=int, default=32)
    ap.add_argument("--cheb-degree", type=int, default=5)
    ap.add_argument("--no-sweep", action="store_true", help="skip the apply sweep and the FP64-MG comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffer) measurement")
    ap.add_argument("--mode", choices=["newton", "apply", "pdas", "loadsteps", "vcycle", "adjoint", "spmv"],
                    default="newton",
                    help="apply: time only the finest-level Jacobian apply (--precision) on the workload; "
                         "pdas: full active-set Newton solve to --newton-rtol, FP64 vs FP32 multigrid; "
                         "spmv: assembled-matrix (cuSPARSE) product against the matrix-free one, p = 1..4")
    ap.add_argument("--state", choices=["random", "tension"], default="random",
                    help="random: seeded u, phi (the apply-sweep workload); tension: u = 0 with the top load "
                         "lifted, phi = 1 except 0 on the slit (a load step from rest)")
    ap.add_argument("--newton-rtol", type=float, default=1e-8)
    ap.add_argument("--load-steps", type=int, default=10, help="--mode loadsteps: number of load steps")
    ap.add_argument("--load-inc", type=float, default=1e-4, help="--mode loadsteps: top displacement increment")
    ap.add_argument("--specimen", choices=["tension", "shear"], default="tension",
                    help="--mode loadsteps: top face pulled up (Sec. 5.1) or moved to the right (Sec. 5.2)")
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket the last timed step (--mode vcycle: one extra cycle) by cudaProfilerStart/Stop, "
                         "for `ncu --profile-from-start off`")
    ap.add_argument("--newton-max", type=int, default=30, help="--mode loadsteps: Newton iterations per load step")
    ap.add_argument("--gmres-max", type=int, default=500, help="--mode loadsteps: FGMRES iterations per linear solve")
    ap.add_argument("--max-seconds", type=float, default=600.0,
                    help="--mode loadsteps: stop a precision's loading after this many seconds (partial result)")
    ap.add_argument("--precision", type=int, default=64, help="precision of --mode apply")
    ap.add_argument("--coarse-precision", type=int, default=64,
                    help="coarse solve of the FP32 multigrid: 64 FP64 inverses (default), 32 FP32 inverses")
    ap.add_argument("--fp32-tangent", type=int, default=0,
                    help="FP32 applies (2D): 0 stored per-point values, 1 recompute the tangent from the nodal state")
    ap.add_argument("--fp64-mode", type=int, default=1,
                    help="FP64 Jacobian applies: 0 native FP64, 1 double-word arithmetic on the FP32 pipe (2D)")
    return ap.parse_args()


def workload_name(a):
    n1 = a.degree * a.cells + 1
    nd = (a.dim + 1) * n1 ** a.dim
    return "%dD Q%d %s notched specimen, %d DoFs, split %s, PDAS Newton step with %s GMG" % (
        a.dim, a.degree, "x".join([str(a.cells)] * a.dim), nd, "miehe" if a.split else "none",
        "FP32 (mixed)" if a.mg_precision == 32 else "FP64")


# ---- multi-rank aggregation (replicas: every rank solves its own copy, no data-path collective) ---
def max_over_ranks(ms, world, device):
    """The slowest rank's step time (ms); world == 1 returns ms unchanged."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(n_dofs_per_rank, world, ms):
    """Whole-job throughput: the DoFs all ranks processed per second of the slowest rank's step."""
    return n_dofs_per_rank * world / (ms * 1e-3)


# ---- measured DRAM traffic of the roofline kernel (from a committed ncu summary) --------------
TRAFFIC_SOURCES = ("pff_op.cuh", "pff_common.cuh", "pff_df64.cuh", "op_jac2_f32.cu", "op_jac3_f32.cu")


def kernel_source_hash():
    """sha256 over the sources of the FP32 Jacobian kernels: a traffic record counts only for them."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2005_00331_gb300", "csrc")
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(a, n_dofs, profiles_dir=None):
    """dram__bytes_read + dram__bytes_write per launch of the FP32 finest-level apply, from a
    'traffic-record:' line of a profiles/*.md summary with the same kernel sources and workload
    family (scaled by DoFs); None when no record matches the current kernel."""
    import glob
    want = {"dim": str(a.dim), "degree": str(a.degree), "split": str(a.split), "source": kernel_source_hash()}
    here = profiles_dir or os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles")
    for fn in sorted(glob.glob(os.path.join(here, "*.md"))):
        with open(fn) as fh:
            for ln in fh:
                if not ln.strip().startswith("traffic-record:"):
                    continue
                kv = dict(x.split("=", 1) for x in ln.split(":", 1)[1].split() if "=" in x)
                if all(kv.get(k) == v for k, v in want.items()):
                    return float(kv["bytes"]) * n_dofs / float(kv["dofs"])
    return None


# ---- synthetic state (inputs module + the library's own node flags) -------------------------
def make_state(ctx, a, seed=0):
    import torch

    from paper_2005_00331_gb300 import PFF_FLAG_SLIT, PFF_FLAG_TOP, inputs
    nn, dim = ctx.n_nodes, a.dim
    fl = ctx.node_flags().cpu().numpy()
    U = np.zeros(ctx.n_dofs)
    if getattr(a, "state", "random") == "tension":
        U[(dim - 1) * nn:dim * nn][(fl & PFF_FLAG_TOP) != 0] = 1e-3
        phi = np.ones(nn)
        phi[(fl & PFF_FLAG_SLIT) != 0] = 0.0
        U[dim * nn:] = phi
        return U, phi.copy()
    dmask = np.concatenate([((fl >> c) & 1).astype(bool) for c in range(dim)])
    U[:dim * nn] = np.where(dmask, 0.0, inputs.displacement_noise(nn, dim, seed, std=1e-3))
    U[(dim - 1) * nn:dim * nn][(fl & PFF_FLAG_TOP) != 0] = 1e-3
    phi = inputs.uniform_phase(nn, seed)
    phi[(fl & PFF_FLAG_SLIT) != 0] = 0.0
    U[dim * nn:] = phi
    phi_old = inputs.phi_old_above(phi, seed)
    return U, phi_old


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    try:
        with open(PEAKS_FILE) as fh:
            p = json.load(fh)
        return p.get("hbm_gbs"), "measured"
    except (OSError, ValueError):
        return 6800.0, "fallback"


def qp_values(dim, split):
    nm = 3 if dim == 2 else 6
    return (2 + nm + 2) if split == 0 else (nm * (nm + 1) // 2 + nm + 2)


def apply_bytes_per_dof(dim, p, split, real_bytes):
    """Algorithmic bytes per DoF of one Jacobian apply with stored per-point data: read x, write y,
    read the per-point data ((p+1)^dim points of qp_values each per cell) and one flag byte per
    node; (d+1) p^d DoFs per cell asymptotically."""
    dofs_per_cell = (dim + 1) * p ** dim
    per_cell = qp_values(dim, split) * (p + 1) ** dim * real_bytes
    return 2 * real_bytes + per_cell / dofs_per_cell + 1.0 / (dim + 1)


def method_bytes_per_dof(dim, real_bytes):
    """Algorithmic (method-minimum) bytes per DoF of one Jacobian apply: read x and write y (one value
    per DoF each), read the nodal state (u, phi, phi~: d + 2 values per node, from which the tangent can
    be recomputed) and one flag byte per node; d + 1 DoFs per node."""
    return 2 * real_bytes + (dim + 2) * real_bytes / (dim + 1) + 1.0 / (dim + 1)


def apply_flops_per_dof(dim, p, split):
    """Floating-point operations per DoF of one Jacobian apply as the kernels k_op2d / k_op3d do it
    (two per fused multiply-add; amortised over large tiles, seams neglected). n = p + 1 points per
    direction; per cell: x-pass, y-pass (3D), fused last-direction pass with the pointwise tangent
    and its transpose, then the transposed passes back to the nodes."""
    n = p + 1
    if dim == 2:
        pw = 20 if split else 12
        fma = 6 * n * n * p + 9 * n ** 3 + 7 * n ** 3 + 6 * n * p * p + pw * n * n
        return 2.0 * fma / (3 * p * p)
    pw = 56 if split else 22
    fma = (8 * n * n * p * p + 12 * p * n ** 3 + 16 * n ** 4 + 13 * n ** 4 + 12 * n * n * p * p + 8 * n * p ** 3
           + pw * n ** 3)
    return 2.0 * fma / (4 * p ** 3)


# ---- native arm ------------------------------------------------------------------------------
def run_native(a, rank, world):
    import torch

    from paper_2005_00331_gb300 import PFF_PROF_JAC32_L0, PFF_PROF_JAC64_L0, PFF_PROF_OFF, launch_count, setup_mesh
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    eps = 2.0 / a.cells
    ctx = setup_mesh(dim=a.dim, degree=a.degree, n_cells_1d=a.cells, split=a.split, eps=eps,
                     mg_precision=a.mg_precision, cheb_degree=a.cheb_degree, fp64_mode=a.fp64_mode,
                     fp32_tangent=a.fp32_tangent)
    U_h, phi_old_h = make_state(ctx, a, seed=rank)
    U = torch.from_numpy(U_h).to(dev)
    phi_old = torch.from_numpy(phi_old_h).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2
    nd = ctx.n_dofs

    def step():
        ctx.set_state(U, phi_old, phi_old, None)
        return ctx.solve_newton_step(check=False)

    prof_family = PFF_PROF_JAC32_L0 if a.mg_precision == 32 else PFF_PROF_JAC64_L0
    ctx.profile(prof_family)  # graphs with timing nodes are captured during the warm-up steps
    for _ in range(a.warmup):
        rep = step()
    torch.cuda.synchronize()
    ctx.profile(prof_family)  # reset the counters: only the timed steps count
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    reps = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    n_launch0 = launch_count()
    with ClockSampler(torch.cuda.current_device()) as clk:
        t0 = time.perf_counter()
        for i in range(a.steps):
            flush.zero_()
            last = a.profile_range and i == a.steps - 1
            if last:
                torch.cuda.synchronize()
                torch.cuda.cudart().cudaProfilerStart()
            ev[i][0].record(stream)
            reps.append(step())
            ev[i][1].record(stream)
            if last:
                torch.cuda.synchronize()
                torch.cuda.cudart().cudaProfilerStop()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
    n_launch = launch_count() - n_launch0
    if world > 1:
        torch.distributed.barrier()
    launches, kern_ms = ctx.profile_result()
    step_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    ms = sum(step_ms) / len(step_ms)
    out = {"step_ms": ms, "wall_ms": (t1 - t0) * 1e3 / a.steps, "reports": reps, "clocks": clk.summary(),
           "kern_launches": launches, "kern_ms": kern_ms, "n_dofs": nd, "launches": n_launch}

    # end to end through the C-ABI with host buffers: H2D of the state, step, D2H of the result
    U_pin = torch.from_numpy(U_h).pin_memory()
    po_pin = torch.from_numpy(phi_old_h).pin_memory()
    U_back = torch.empty(nd, dtype=torch.float64).pin_memory()
    U_d = torch.empty(nd, dtype=torch.float64, device=dev)
    po_d = torch.empty_like(phi_old)
    e2e = []
    for i in range(0 if a.no_e2e else a.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        U_d.copy_(U_pin, non_blocking=True)
        po_d.copy_(po_pin, non_blocking=True)
        ctx.set_state(U_d, po_d, po_d, None)
        ctx.solve_newton_step(U_out=U_d, check=False)
        U_back.copy_(U_d, non_blocking=True)
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t)
    # same statistic as the device-timed value, through the same graphs (with the timing nodes the
    # roofline reads: the e2e steps run exactly the code of the timed steps, plus the copies)
    out["e2e_s"] = statistics.mean(e2e) if e2e else float("nan")
    ctx.profile(PFF_PROF_OFF)
    out["h2d"] = 8 * (nd + ctx.n_nodes)
    out["d2h"] = 8 * nd

    if not a.no_sweep and rank == 0:
        out["sweep"] = apply_sweep(a, dev, flush)
        # the same Newton step with the FP64 multigrid
        ctx64 = setup_mesh(dim=a.dim, degree=a.degree, n_cells_1d=a.cells, split=a.split, eps=eps,
                           mg_precision=64, cheb_degree=a.cheb_degree, fp64_mode=0)
        ctx64.set_state(U, phi_old, phi_old, None)
        ctx64.solve_newton_step(check=False)
        t64 = []
        rep64 = None
        for _ in range(2):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx64.set_state(U, phi_old, phi_old, None)
            rep64 = ctx64.solve_newton_step(check=False)
            e1.record(stream)
            torch.cuda.synchronize()
            t64.append(e0.elapsed_time(e1))
        # agreement of the two Newton updates
        Um = ctx.get_state()
        ctx.set_state(U, phi_old, phi_old, None)
        ctx.solve_newton_step(check=False)
        Um = ctx.get_state()
        U64 = ctx64.get_state()
        out["fp64_mg"] = {"step_ms": min(t64), "gmres_iters": rep64["gmres_iters"], "status": rep64["status"],
                          "rel_diff_vs_mixed": float((Um - U64).norm() / (U64 - U).norm())}
        ctx64.close()
        out["pdas_1e8"], out["pdas_finals"] = pdas_to_tolerance(a, dev, U_h, phi_old_h)
        out["phi_old_h"] = phi_old_h
    ctx.close()
    return out


def oracle_specimen(dim, p, N, split, state):
    """The specimen of the workload as the oracle builds it (its own mesh, Dirichlet lift and slit), fed
    from the seeded input generators: (mesh, params, U, phi_old)."""
    from oracle import fe, mesh as M
    from paper_2005_00331_gb300 import inputs
    m = M.Mesh(dim, p, N)
    prm = fe.Params(eps=2.0 / N, split=split)
    nn = m.n_nodes
    U = m.dirichlet_values(1e-3)
    if state == "tension":
        phi = np.ones(nn)
        phi[m.slit_nodes()] = 0.0
        U[dim * nn:] = phi
        return m, prm, U, phi.copy()
    U[:dim * nn] += np.where(m.dirichlet_mask()[:dim * nn], 0.0, inputs.displacement_noise(nn, dim, 0))
    phi = inputs.uniform_phase(nn, 0)
    phi[m.slit_nodes()] = 0.0
    U[dim * nn:] = phi
    return m, prm, U, inputs.phi_old_above(phi, 0)


ORACLE_CHECK_CASES = ((2, 1, 32, "tension"), (2, 2, 64, "random"))


def oracle_errors(a, dev):
    """Error of the GPU's Newton update against the oracle's (one step of Alg. 1 with a sparse direct
    solve), with the mixed multigrid (double-word outer operator, as timed) and with the FP64 one (native
    FP64 outer operator): ||U_gpu - U_oracle|| / ||U_oracle - U||, and whether the active sets agree
    bit for bit. Sizes the oracle finishes in seconds: the 32 x 32 Q1 tension test from rest and the
    2D Q2 64 x 64 random state of the workload family. The linear solves stop at relative 1e-6."""
    import torch

    from oracle import solvers as S
    from paper_2005_00331_gb300 import setup_mesh
    out = {}
    for dim, p, N, state in ORACLE_CHECK_CASES:
        m, prm, U, po = oracle_specimen(dim, p, N, state=state, split=a.split)
        U_ref, act_ref, _, _ = S.pdas_step(m, prm, U, po, po)
        step = float(np.linalg.norm(U_ref - U))
        case = {"n_dofs": m.n_dofs, "state": state, "active": int(act_ref.sum())}
        for name, mg, fm in (("mixed", 32, 1), ("fp64", 64, 0)):
            with setup_mesh(dim=dim, degree=p, n_cells_1d=N, split=a.split, eps=2.0 / N, mg_precision=mg,
                            cheb_degree=a.cheb_degree, fp64_mode=fm) as ctx:
                t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
                ctx.set_state(t(U), t(po), t(po), None)
                rep = ctx.solve_newton_step(check=False)
                Ug = ctx.get_state().cpu().numpy()
                act = ctx.get_active().cpu().numpy().astype(bool)
            case[name] = {"rel_err_update": float(np.linalg.norm(Ug - U_ref)) / step,
                          "active_set_equal": bool(np.array_equal(act, act_ref)), "gmres_iters": rep["gmres_iters"],
                          "gmres_rel": rep["gmres_rel"]}
        out["%dD_Q%d_%d" % (dim, p, N)] = case
    return out


def pdas_to_tolerance(a, dev, U_h, po_h, rtol=1e-8):
    """The full active-set Newton solve of the workload (Alg. 1 until the active set is unchanged and
    ||R~|| <= rtol ||R~_0||) with the mixed multigrid (FP32 levels, FP64 coarse solve, double-word outer
    operator, as timed) and with the plain FP64 one (FP64 multigrid, native FP64 outer operator): time
    per Newton step (CUDA events, after a warm-up solve), Newton and FGMRES iterations, and the final
    reduced residual recomputed by the oracle at the GPU's final state (Dirichlet and final active rows
    removed) relative to the loop's ||R~_0||."""
    import torch

    from paper_2005_00331_gb300 import setup_mesh
    stream = torch.cuda.current_stream()
    out, finals = {"newton_rtol": rtol}, {}
    U = torch.from_numpy(U_h).to(dev)
    po = torch.from_numpy(po_h).to(dev)
    # mixed_native_outer separates the two changes between "mixed" and "fp64": the multigrid precision and
    # the outer operator's arithmetic (double-word vs native FP64)
    for name, mg, fm in (("mixed", 32, a.fp64_mode), ("mixed_native_outer", 32, 0), ("fp64", 64, 0)):
        with setup_mesh(dim=a.dim, degree=a.degree, n_cells_1d=a.cells, split=a.split, eps=2.0 / a.cells,
                        mg_precision=mg, cheb_degree=a.cheb_degree, fp64_mode=fm,
                        fp32_tangent=a.fp32_tangent) as ctx:
            ctx.set_state(U, po, po, None)
            ctx.solve_pdas(max_iters=30, newton_rtol=rtol, check=False)  # warm-up: graph capture
            ctx.set_state(U, po, po, None)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st, reps = ctx.solve_pdas(max_iters=30, newton_rtol=rtol, check=False)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            Uf = ctx.get_state().cpu().numpy()
            act = ctx.get_active().cpu().numpy().astype(bool)
        finals[name] = (Uf, act)
        out[name] = {"status": st, "newton_steps": len(reps), "ms": ms, "ms_per_newton_step": ms / max(1, len(reps)),
                     "gmres_iters": [r["gmres_iters"] for r in reps], "res_norm_0": reps[0]["res_norm"],
                     "res_rel_last_step": reps[-1]["res_norm"] / reps[0]["res_norm"],
                     "n_active": reps[-1]["n_active"]}
    out["rel_diff_mixed_vs_fp64"] = float(np.linalg.norm(finals["mixed"][0] - finals["fp64"][0]) /
                                          np.linalg.norm(finals["fp64"][0] - U_h))
    out["speedup_mixed_vs_fp64"] = out["fp64"]["ms_per_newton_step"] / out["mixed"]["ms_per_newton_step"]
    out["speedup_mixed_native_outer_vs_fp64"] = (out["fp64"]["ms_per_newton_step"] /
                                                 out["mixed_native_outer"]["ms_per_newton_step"])
    return out, finals


def oracle_final_residuals(a, po_h, finals, pdas):
    """The final reduced residual of each 1e-8 solve recomputed by the oracle at the GPU's final state
    (Dirichlet rows and the final active set removed), relative to the loop's ||R~_0||."""
    from oracle import fe
    m, prm, _, _ = oracle_specimen(a.dim, a.degree, a.cells, a.split, "random")
    for name, (Uf, act) in finals.items():
        R = fe.residual(m, prm, Uf, po_h)
        R[a.dim * m.n_nodes:][act] = 0.0
        pdas[name]["oracle_final_res_rel"] = float(np.linalg.norm(R)) / pdas[name]["res_norm_0"]


def apply_sweep(a, dev, flush, reps=20):
    """Jacobian apply at p = 1..4 on the 2D 256^2 mesh, FP64 and FP32, L2 flushed before each."""
    import torch

    from paper_2005_00331_gb300 import setup_mesh
    res = {}
    stream = torch.cuda.current_stream()
    for p in (1, 2, 3, 4):
        b = argparse.Namespace(**vars(a))
        b.degree = p
        ctx = setup_mesh(dim=a.dim, degree=p, n_cells_1d=a.cells, split=a.split, eps=2.0 / a.cells,
                         mg_precision=32, fp64_mode=0)
        ctxdf = setup_mesh(dim=a.dim, degree=p, n_cells_1d=a.cells, split=a.split, eps=2.0 / a.cells,
                           mg_precision=32, fp64_mode=1)
        U_h, po_h = make_state(ctx, b, seed=0)
        U = torch.from_numpy(U_h).to(dev)
        po = torch.from_numpy(po_h).to(dev)
        nn = ctx.n_nodes
        act = (po - U[a.dim * nn:] < 1e-8).to(torch.uint8)  # the configured rule: phi_old - phi < 1e-8
        ctx.set_state(U, po, po, act.contiguous())
        ctxdf.set_state(U, po, po, act.contiguous())
        for name, cx, prec, dt in (("fp64", ctx, 64, torch.float64), ("fp64ff", ctxdf, 64, torch.float64),
                                   ("fp32", ctx, 32, torch.float32)):
            x = torch.randn(ctx.n_dofs, dtype=torch.float64, device=dev).to(dt)
            y = torch.empty_like(x)
            for _ in range(3):
                cx.apply_jacobian(x, y)
            times = []
            for _ in range(reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                cx.apply_jacobian(x, y)
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            med = statistics.median(times)
            nbytes = apply_bytes_per_dof(a.dim, p, a.split, 8 if prec == 64 else 4) * ctx.n_dofs
            flops = apply_flops_per_dof(a.dim, p, a.split) * ctx.n_dofs
            res["p%d_%s" % (p, name)] = {
                "dofs": ctx.n_dofs, "median_ms": med, "best_ms": min(times),
                "dofs_per_s": ctx.n_dofs / (med * 1e-3), "GB_per_s": nbytes / (med * 1e-3) / 1e9,
                "TFLOP_per_s": flops / (med * 1e-3) / 1e12}
        ctx.close()
        ctxdf.close()
    return res


def run_apply_only(a):
    """K finest-level Jacobian applies (full mode, masked) after W warm-up applies, each timed with
    CUDA events after an L2 flush."""
    import torch

    from paper_2005_00331_gb300 import launch_count, setup_mesh
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    ctx = setup_mesh(dim=a.dim, degree=a.degree, n_cells_1d=a.cells, split=a.split, eps=2.0 / a.cells,
                     mg_precision=32, fp64_mode=a.fp64_mode,
                     fp32_tangent=a.fp32_tangent)
    U_h, po_h = make_state(ctx, a, seed=0)
    U = torch.from_numpy(U_h).to(dev)
    po = torch.from_numpy(po_h).to(dev)
    nn = ctx.n_nodes
    act = (po - U[a.dim * nn:] < 1e-8).to(torch.uint8).contiguous()
    ctx.set_state(U, po, po, act)
    dt = torch.float64 if a.precision == 64 else torch.float32
    x = torch.randn(ctx.n_dofs, dtype=torch.float64, device=dev).to(dt)
    y = torch.empty_like(x)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(a.warmup):
        ctx.apply_jacobian(x, y)
    torch.cuda.synchronize()
    n0 = launch_count()
    times = []
    for _ in range(a.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.apply_jacobian(x, y)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    med = statistics.median(times)
    nd = ctx.n_dofs
    real = 8 if a.precision == 64 else 4
    return {"mode": "apply", "dofs": nd, "precision": a.precision, "median_ms": med, "best_ms": min(times),
            "dofs_per_s": nd / (med * 1e-3),
            "GB_per_s": apply_bytes_per_dof(a.dim, a.degree, a.split, real) * nd / (med * 1e-3) / 1e9,
            "TFLOP_per_s": apply_flops_per_dof(a.dim, a.degree, a.split) * nd / (med * 1e-3) / 1e12,
            "launches": launch_count() - n0}


def _event_times(fn, steps, warmup, flush, stream):
    """CUDA-event durations (ms) of `steps` calls of fn after `warmup` untimed ones, L2 flushed before each."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return times


def run_spmv(a):
    """The paper's SpMV-vs-MFMV comparison over the polynomial degree (Sec. 6.3, fig. compare:vmult):
    for p = 1..4 on the --dim/--cells specimen, the masked Jacobian of the workload state assembled
    into CSR (pff_csr_assemble; assembly time reported, not part of the product) and multiplied by
    cuSPARSE, against the matrix-free FP64 apply (--fp64-mode) and the FP32 one; best and median of
    --steps event-timed products after --warmup, the L2 flushed before each."""
    import torch

    from paper_2005_00331_gb300 import setup_mesh
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    hbm, hbm_kind = peaks()
    out = {"mode": "spmv", "dim": a.dim, "cells_per_dir": a.cells, "split": a.split, "fp64_mode": a.fp64_mode,
           "steps": a.steps, "warmup": a.warmup, "hbm_peak_GB_per_s": hbm, "hbm_peak_kind": hbm_kind, "degrees": {}}
    for p in (1, 2, 3, 4):
        b = argparse.Namespace(**vars(a))
        b.degree = p
        ctx = setup_mesh(dim=a.dim, degree=p, n_cells_1d=a.cells, split=a.split, eps=2.0 / a.cells,
                         mg_precision=32, fp64_mode=a.fp64_mode)
        U_h, po_h = make_state(ctx, b, seed=0)
        U = torch.from_numpy(U_h).to(dev)
        po = torch.from_numpy(po_h).to(dev)
        act = (po - U[a.dim * ctx.n_nodes:] < 1e-8).to(torch.uint8).contiguous()
        ctx.set_state(U, po, po, act)
        t0 = time.perf_counter()
        nnz = ctx.csr_assemble()
        t_asm = time.perf_counter() - t0
        nd = ctx.n_dofs
        x = torch.randn(nd, dtype=torch.float64, device=dev)
        y = torch.empty_like(x)
        x32, y32 = x.float(), torch.empty(nd, dtype=torch.float32, device=dev)
        t_sp = _event_times(lambda: ctx.csr_spmv(x, y), a.steps, a.warmup, flush, stream)
        y_sp = y.clone()
        t_mf = _event_times(lambda: ctx.apply_jacobian(x, y), a.steps, a.warmup, flush, stream)
        t_mf32 = _event_times(lambda: ctx.apply_jacobian(x32, y32, precision=32), a.steps, a.warmup, flush, stream)
        diff = float((y_sp - y).norm() / max(float(y.norm()), 1e-300))
        sp_bytes = nnz * 12 + (nd + 1) * 4 + 2 * nd * 8  # values + column indices, row offsets, x and y once
        best = min(t_sp)
        out["degrees"][str(p)] = {
            "n_dofs": nd, "nnz": nnz, "nnz_per_row": nnz / nd, "csr_MB": (nnz * 12 + (nd + 1) * 4) / 1e6,
            "assemble_s": t_asm, "spmv_best_ms": best, "spmv_median_ms": statistics.median(t_sp),
            "mf64_best_ms": min(t_mf), "mf64_median_ms": statistics.median(t_mf),
            "mf32_best_ms": min(t_mf32), "mf32_median_ms": statistics.median(t_mf32),
            "spmv_GB_per_s": sp_bytes / (best * 1e-3) / 1e9,
            "spmv_frac_of_hbm": sp_bytes / (best * 1e-3) / 1e9 / hbm if hbm else None,
            "mf64_speedup_vs_spmv": best / min(t_mf), "rel_diff_spmv_vs_mf64": diff}
        print("p=%d: %s" % (p, json.dumps(out["degrees"][str(p)])), file=sys.stderr, flush=True)
        ctx.close()
    return out


def run_pdas(a):
    """Full active-set Newton solve (Alg. 1 to --newton-rtol) from the workload state, with the FP32
    (mixed) and with the FP64 multigrid; both inside FP64 FGMRES with the FP64 residual."""
    import torch

    from paper_2005_00331_gb300 import setup_mesh
    dev = torch.device("cuda", torch.cuda.current_device())
    out = {"mode": "pdas", "workload": workload_name(a), "state": a.state, "newton_rtol": a.newton_rtol,
           "coarse_precision_of_fp32_mg": a.coarse_precision}
    finals = {}
    for prec in (32, 64):
        ctx = setup_mesh(dim=a.dim, degree=a.degree, n_cells_1d=a.cells, split=a.split, eps=2.0 / a.cells,
                         mg_precision=prec, cheb_degree=a.cheb_degree, fp64_mode=a.fp64_mode,
                         coarse_precision=a.coarse_precision)
        U_h, po_h = make_state(ctx, a, seed=0)
        U = torch.from_numpy(U_h).to(dev)
        po = torch.from_numpy(po_h).to(dev)
        # warm-up solve (graph capture, kernel attributes), then the timed solve from the same state
        ctx.set_state(U, po, po, None)
        ctx.solve_pdas(max_iters=30, newton_rtol=a.newton_rtol, check=False)
        ctx.set_state(U, po, po, None)
        torch.cuda.synchronize()
        t = time.perf_counter()
        st, reps = ctx.solve_pdas(max_iters=30, newton_rtol=a.newton_rtol, check=False)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        finals[prec] = ctx.get_state()
        out["mg_fp%d" % prec] = {
            "status": st, "newton_steps": len(reps), "seconds": dt, "s_per_newton_step": dt / max(1, len(reps)),
            "gmres_iters": [r["gmres_iters"] for r in reps], "res_norms": [r["res_norm"] for r in reps],
            "n_active_final": reps[-1]["n_active"] if reps else None}
        out["n_dofs"] = ctx.n_dofs
        ctx.close()
    d = (finals[32] - finals[64]).norm() / max(float(finals[64].norm()), 1e-300)
    out["rel_diff_mixed_vs_fp64"] = float(d)
    return out


def run_adjoint(a):
    """Residual under torch.autograd with the hand-written adjoint: forward R(U; G_c, lambda, mu) and
    backward (transpose Jacobian apply + nodal parameter gradients) for a seeded lognormal G_c field,
    --steps timed passes after --warmup (CUDA events)."""
    import torch

    from paper_2005_00331_gb300 import ResidualFunction, inputs, setup_mesh
    dev = torch.device("cuda", torch.cuda.current_device())
    ctx = setup_mesh(dim=a.dim, degree=a.degree, n_cells_1d=a.cells, split=a.split, eps=2.0 / a.cells,
                     mg_precision=a.mg_precision, fp64_mode=a.fp64_mode)
    U_h, po_h = make_state(ctx, a, seed=0)
    nn = ctx.n_nodes
    U = torch.from_numpy(U_h).to(dev).requires_grad_(True)
    po = torch.from_numpy(po_h).to(dev)
    gc = torch.from_numpy(inputs.lognormal_field(nn, 0)).to(dev).requires_grad_(True)
    lam = torch.full((nn,), 121.15, dtype=torch.float64, device=dev, requires_grad=True)
    mu = torch.full((nn,), 80.77, dtype=torch.float64, device=dev, requires_grad=True)
    v = torch.from_numpy(inputs.normal_vector(ctx.n_dofs, 1)).to(dev)

    def step():
        R = ResidualFunction.apply(ctx, U, po, po, gc, lam, mu)
        return torch.autograd.grad((R * v).sum(), (U, gc, lam, mu))

    for _ in range(max(a.warmup, 1)):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    return {"mode": "adjoint", "workload": workload_name(a).split(", PDAS")[0] + ", FP64 residual + adjoint",
            "n_dofs": ctx.n_dofs, "ms_per_forward_backward": ms, "dofs_per_s": ctx.n_dofs / (ms * 1e-3),
            "passes": a.steps}


def run_vcycle(a):
    """The FP32 (or FP64, --mg-precision) V-cycle of the workload's first Newton step, replayed
    --steps times after --warmup replays (CUDA events, warm caches)."""
    import torch

    from paper_2005_00331_gb300 import setup_mesh
    dev = torch.device("cuda", torch.cuda.current_device())
    ctx = setup_mesh(dim=a.dim, degree=a.degree, n_cells_1d=a.cells, split=a.split, eps=2.0 / a.cells,
                     mg_precision=a.mg_precision, cheb_degree=a.cheb_degree, fp64_mode=a.fp64_mode,
                     fp32_tangent=a.fp32_tangent)
    U_h, po_h = make_state(ctx, a, seed=0)
    ctx.set_state(torch.from_numpy(U_h).to(dev), torch.from_numpy(po_h).to(dev),
                  torch.from_numpy(po_h).to(dev), None)
    ctx.solve_newton_step(check=False)
    r = torch.randn(ctx.n_dofs, dtype=torch.float64, device=dev)
    z = torch.empty_like(r)
    for _ in range(max(a.warmup, 1)):
        ctx.vcycle(r, z)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        ctx.vcycle(r, z)
    e1.record()
    torch.cuda.synchronize()
    if a.profile_range:
        torch.cuda.cudart().cudaProfilerStart()
        ctx.vcycle(r, z)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
    return {"mode": "vcycle", "workload": workload_name(a), "levels": ctx.n_levels,
            "ms_per_cycle": e0.elapsed_time(e1) / a.steps, "replays": a.steps}


def run_loadsteps(a):
    """Quasi-static loading from rest: --load-steps steps of --load-inc on the top face, each a full
    active-set Newton solve with the extrapolated phase field; FP32 (mixed) vs FP64 multigrid; the top
    face pulled up (--specimen tension, Sec. 5.1) or moved to the right (shear, Sec. 5.2). Each step
    also records the force on the top face in the loading direction (the load-displacement curve)."""
    import torch

    from paper_2005_00331_gb300 import setup_mesh
    dev = torch.device("cuda", torch.cuda.current_device())
    b = argparse.Namespace(**vars(a))
    b.state = "tension"
    out = {"mode": "loadsteps", "workload": workload_name(a), "specimen": a.specimen, "load_steps": a.load_steps,
           "load_inc": a.load_inc, "newton_rtol": a.newton_rtol}
    finals = {}
    for prec in (32, 64):
        ctx = setup_mesh(dim=a.dim, degree=a.degree, n_cells_1d=a.cells, split=a.split, eps=2.0 / a.cells,
                         mg_precision=prec, cheb_degree=a.cheb_degree, fp64_mode=a.fp64_mode,
                         gmres_max_iters=a.gmres_max, coarse_precision=a.coarse_precision)
        U_h, po_h = make_state(ctx, b, seed=0)
        U = torch.from_numpy(U_h).to(dev)
        po = torch.from_numpy(po_h).to(dev)
        U[(a.dim - 1) * ctx.n_nodes:a.dim * ctx.n_nodes] = 0.0  # start from rest: no load yet
        if a.specimen == "shear":
            ctx.set_load_component(0)
        # warm-up: one load step (graph capture, kernel attributes), then restart from rest
        ctx.set_state(U, po, po, None)
        ctx.solve_load_step(a.load_inc, check=False)
        ctx.set_state(U, po, po, None)
        torch.cuda.synchronize()
        t = time.perf_counter()
        steps, newton, iters, status = [], 0, 0, 0
        for k in range(1, a.load_steps + 1):
            t0 = time.perf_counter()
            st, reps = ctx.solve_load_step(k * a.load_inc, max_iters=a.newton_max, newton_rtol=a.newton_rtol,
                                           check=False)
            sec = time.perf_counter() - t0
            steps.append({"load": k * a.load_inc, "status": st, "newton_steps": len(reps),
                          "gmres_iters": [r["gmres_iters"] for r in reps], "seconds": sec,
                          "n_active": reps[-1]["n_active"] if reps else None,
                          "reaction_force": ctx.reaction_force()})  # the load-displacement curve
            print("fp%d load step %d: %s" % (prec, k, json.dumps(steps[-1])), file=sys.stderr, flush=True)
            newton += len(reps)
            status = status or st
            if time.perf_counter() - t > a.max_seconds:
                break
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        finals[prec] = ctx.get_state()
        out["mg_fp%d" % prec] = {"status": status, "seconds": dt, "newton_steps": newton, "load_steps_done": len(steps),
                                 "s_per_newton_step": dt / max(1, newton), "steps": steps}
        out["n_dofs"] = ctx.n_dofs
        ctx.close()
    same = out["mg_fp32"]["load_steps_done"] == out["mg_fp64"]["load_steps_done"]
    out["rel_diff_mixed_vs_fp64"] = (float((finals[32] - finals[64]).norm() / max(float(finals[64].norm()), 1e-300))
                                     if same else None)
    return out


# ---- CPU oracle baseline ----------------------------------------------------------------------
# Cells per direction of the oracle's timed step: the reference arm times one step per benchmark step
# (32^2: ~1-1.5 s each, so that --steps 50 ends within minutes); the cpu_baseline of the GPU line is
# one larger sample (96^2, 112 k DoFs: ~10-15 s of CPU work). The oracle's DoF/s hardly depends on
# the size (32^2, 64^2, 96^2 within 3 % of each other).
CPU_SAMPLE_CELLS = 32
CPU_BASELINE_CELLS = 96


def _oracle_step_code(a, cells, go=None):
    """Source of a process that times one oracle PDAS Newton step (FGMRES + V-cycle, sparse direct
    coarse solve) on the specimen with `cells` cells per direction and prints n_dofs, the step's
    seconds and its wall-clock start and end; with `go` (a time.time() value) the step waits until
    then, so that concurrent processes start together after their imports and set-up."""
    return r"""
import json, sys, time
sys.path.insert(0, %r)
import numpy as np
import importlib.util
from oracle import fe, mesh as M, solvers as S
# the seeded input generators alone (numpy only), without the package and the torch import it makes
spec = importlib.util.spec_from_file_location("pff_inputs", %r)
inputs = importlib.util.module_from_spec(spec)
spec.loader.exec_module(inputs)
dim, p, N, split = %d, %d, %d, %d
m = M.Mesh(dim, p, N)
prm = fe.Params(eps=2.0 / N, split=split)
nn = m.n_nodes
U = m.dirichlet_values(1e-3)
U[:dim * nn] += np.where(m.dirichlet_mask()[:dim * nn], 0.0, inputs.displacement_noise(nn, dim, 0))
phi = inputs.uniform_phase(nn, 0)
phi[m.slit_nodes()] = 0.0
U[dim * nn:] = phi
po = inputs.phi_old_above(phi, 0)
go = %r
if go is not None and go > time.time():
    time.sleep(go - time.time())
w0 = time.time()
t = time.perf_counter()
S.pdas_step(m, prm, U, po, po, solve="gmg", levels_kw=dict(cheb_degree=%d))
dt = time.perf_counter() - t
print(json.dumps({"n_dofs": m.n_dofs, "seconds": dt, "start": w0, "end": time.time()}))
""" % (ROOT, os.path.join(ROOT, "paper_2005_00331_gb300", "inputs.py"), a.dim, a.degree, cells, a.split, go,
       a.cheb_degree)


ORACLE_ENV = dict(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")


def cpu_oracle_sample(a, cells=CPU_SAMPLE_CELLS):
    """Times the oracle's PDAS Newton step on the same specimen family with `cells` cells per
    direction, in one single-threaded process."""
    env = dict(os.environ, **ORACLE_ENV)
    r = subprocess.run([sys.executable, "-c", _oracle_step_code(a, cells)], capture_output=True, text=True, env=env,
                       timeout=600)
    if r.returncode != 0:
        return {"error": r.stderr[-400:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": d["n_dofs"] / d["seconds"], "unit": "DoF/s", "cores": 1, "kind": "oracle",
            "sample": "one oracle PDAS Newton step (FGMRES + GMG) on the %dD Q%d notched specimen with %d^%d "
                      "cells (%d DoFs), %.1f s" % (a.dim, a.degree, cells, a.dim, d["n_dofs"],
                                                   d["seconds"]),
            "host": host_cpu()}


def cpu_oracle_all_cores(a, cells=CPU_SAMPLE_CELLS):
    """The oracle on every host core at once: one single-threaded process per core, each timing one
    step; the throughput is the DoFs of all steps over the span from the first start to the last end
    (process start-up and imports excluded: the steps wait for a common start time)."""
    n = os.cpu_count() or 1
    env = dict(os.environ, **ORACLE_ENV)
    code = _oracle_step_code(a, cells, go=time.time() + 8.0)
    procs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                              env=env) for _ in range(n)]
    outs = []
    for pr in procs:
        try:
            out, err = pr.communicate(timeout=900)
        except subprocess.TimeoutExpired:
            pr.kill()
            out, err = pr.communicate()
        if pr.returncode != 0:
            return {"error": (err or "")[-400:]}
        outs.append(json.loads(out.strip().splitlines()[-1]))
    span = max(d["end"] for d in outs) - min(d["start"] for d in outs)
    dofs = sum(d["n_dofs"] for d in outs)
    return {"value": dofs / span, "unit": "DoF/s", "cores": n, "kind": "oracle",
            "sample": "%d concurrent single-threaded oracle PDAS Newton steps (one per core) on the %dD Q%d notched "
                      "specimen with %d^%d cells, %.1f s from the first start to the last end"
                      % (n, a.dim, a.degree, cells, a.dim, span),
            "host": host_cpu()}


def host_cpu():
    """CPU model and core count of this host (lscpu, else /proc/cpuinfo, else the machine type)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    import platform
    return {"cpu": model or platform.machine(), "nproc": os.cpu_count()}


# ---- main --------------------------------------------------------------------------------------
def main():
    a = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    config = {"workload": workload_name(a), "dim": a.dim, "degree": a.degree, "cells_per_dir": a.cells,
              "split": "miehe" if a.split else "none", "mg_precision": a.mg_precision,
              "cheb_degree": a.cheb_degree, "linear_rtol": 1e-6,
              "fp32_tangent": "recomputed from the nodal state" if a.fp32_tangent else "stored per-point values", "parallelism": "replicas" if world > 1 else "1 GPU",
              "l2": "256 MB buffer written before every timed step (flushes the 135 MB L2)"}
    if a.impl == "reference":
        if rank != 0:
            return
        for _ in range(a.warmup):  # untimed samples (the process start-up and imports they include)
            cpu_oracle_sample(a)
        t = time.perf_counter()
        vals = []
        for _ in range(a.steps):
            c = cpu_oracle_sample(a)
            if "error" in c:
                print(json.dumps({"impl": "reference", "unavailable": "oracle failed: " + c["error"][-200:]}))
                return
            vals.append(c)
        v = statistics.median([c["value"] for c in vals])
        config["sample"] = ("each step times one oracle PDAS Newton step on the %dD Q%d specimen with %d^%d cells "
                            "(%s); the oracle's DoF/s varies by under 3 %% between 32^2 and 96^2 cells"
                            % (a.dim, a.degree, CPU_SAMPLE_CELLS, a.dim, vals[0]["sample"].split("(")[-1].split(")")[0]))
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "DoF/s", "n_gpus": a.gpus,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": (time.perf_counter() - t) * 1e3 / a.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": config,
                "cpu_baseline": {"value": v, "unit": "DoF/s", "cores": 1, "kind": "oracle", "sample": vals[0]["sample"]},
                "e2e": {"value": v, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    if a.mode == "apply":
        torch.cuda.set_device(local if world > 1 else 0)
        print(json.dumps(run_apply_only(a)))
        return
    if a.mode == "pdas":
        torch.cuda.set_device(local if world > 1 else 0)
        print(json.dumps(run_pdas(a)))
        return
    if a.mode == "loadsteps":
        torch.cuda.set_device(local if world > 1 else 0)
        print(json.dumps(run_loadsteps(a)))
        return
    if a.mode == "vcycle":
        torch.cuda.set_device(local if world > 1 else 0)
        print(json.dumps(run_vcycle(a)))
        return
    if a.mode == "adjoint":
        torch.cuda.set_device(local if world > 1 else 0)
        print(json.dumps(run_adjoint(a)))
        return
    if a.mode == "spmv":
        torch.cuda.set_device(local if world > 1 else 0)
        print(json.dumps(run_spmv(a)))
        return
    if world > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    r = run_native(a, rank, world)
    ms = max_over_ranks(r["step_ms"], world, "cuda")
    value = job_value(r["n_dofs"], world, ms)
    if rank != 0:
        torch.distributed.destroy_process_group()
        return
    hbm, hbm_kind = peaks()
    real_bytes = 4 if a.mg_precision == 32 else 8
    per_launch = r["kern_ms"] / max(1, r["kern_launches"])
    bpd = method_bytes_per_dof(a.dim, real_bytes)
    achieved = bpd * r["n_dofs"] / (per_launch * 1e-3) / 1e9 if r["kern_launches"] else None
    rep = r["reports"][-1]
    line = {
        "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": ("f64 outer (%s) / f32 multigrid" % ("double-word on FP32 pipe" if a.fp64_mode else "native")
                  if a.mg_precision == 32 else "f64"), "data": "synthetic",
        "config": config,
        "newton": {"gmres_iters": rep["gmres_iters"], "gmres_rel": rep["gmres_rel"], "status": rep["status"],
                   "n_active": rep["n_active"], "res_norm": rep["res_norm"],
                   "t_residual_ms": rep["t_residual_ms"], "t_setup_ms": rep["t_setup_ms"],
                   "t_solve_ms": rep["t_solve_ms"], "wall_ms_per_step": r["wall_ms"]},
        "roofline": {"kernel": "%s Jacobian apply, FP%d, finest level, inside the timed steps" % (
            "k_jac2_staged" if a.dim == 2 else "k_op3d", real_bytes * 8),
                     "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": (achieved / hbm) if achieved else None,
                     "traffic": measured_traffic(a, r["n_dofs"]) if a.mg_precision == 32 else None,
                     "peak_kind": hbm_kind, "launches": r["kern_launches"], "avg_launch_ms": per_launch,
                     "bytes_per_dof": bpd, "bytes_kind": "method minimum: x, y, nodal state (u, phi, phi~), flags",
                     "stored_tangent_bytes_per_dof": apply_bytes_per_dof(a.dim, a.degree, a.split, real_bytes)},
        "e2e": {"value": r["n_dofs"] * world / r["e2e_s"], "unit": "DoF/s", "h2d_bytes_per_step": r["h2d"],
                "d2h_bytes_per_step": r["d2h"]},
        "clocks": r["clocks"],
        "gpu_launches": r["launches"],
    }
    if "sweep" in r:
        line["jacobian_apply"] = r["sweep"]
        line["fp64_mg_newton_step"] = r["fp64_mg"]
        line["pdas_1e8"] = r["pdas_1e8"]
        fp64 = r["sweep"].get("p%d_fp64" % a.degree)
        if fp64:
            line["jacobian_apply_fp64_roofline"] = {
                "kernel": "native FP64 arithmetic", "bound": "alu", "achieved": fp64["TFLOP_per_s"],
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": fp64["TFLOP_per_s"] / FP64_PEAK_TFLOPS,
                "peak_kind": "derived: 152 SMs x 2 FP64 FMA/clk x 2 x 2.07 GHz"}
        ff = r["sweep"].get("p%d_fp64ff" % a.degree)
        if ff:
            line["jacobian_apply_fp64ff_roofline"] = {
                "kernel": "FP64 values, double-word arithmetic on the FP32 pipe", "bound": "hbm",
                "achieved": ff["GB_per_s"], "peak": hbm, "unit": "GB/s", "frac": ff["GB_per_s"] / hbm,
                "peak_kind": hbm_kind}
    if not a.no_cpu and world == 1:  # rank 0 at N = 1 only: the oracle's timings and checks
        if "pdas_finals" in r:
            oracle_final_residuals(a, r["phi_old_h"], r["pdas_finals"], line["pdas_1e8"])
            line["oracle_error"] = oracle_errors(a, torch.device("cuda", torch.cuda.current_device()))
        for key, fn in (("cpu_baseline", lambda: cpu_oracle_sample(a, CPU_BASELINE_CELLS)),
                        ("cpu_baseline_all_cores", lambda: cpu_oracle_all_cores(a))):
            try:  # the CPU baselines are reported beside the GPU numbers; they must not lose the line
                line[key] = fn()
            except (OSError, ValueError, KeyError, subprocess.SubprocessError) as e:
                line[key] = {"error": "%s: %s" % (type(e).__name__, e)}
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
