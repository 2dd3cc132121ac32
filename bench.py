"""Benchmark: FP64 SIPG operator throughput inside a Jacobi-PCG Poisson solve.

Workload (one step): the pressure Poisson problem on the tanh-graded channel
2 pi x 2 x pi with 32^3 cells, gamma = 1.8, periodic in x and z, Dirichlet
walls, k = 4 (4,096,000 DoF); right-hand side b = M f_I with
f = (5 + pi^2/4) sin x cos(pi y/2) sin 2z at the nodes; Jacobi-preconditioned
CG from x = 0 to a relative residual of 1e-10, one CUDA graph per 16
iterations.  The step is the whole solve, in native FP64 arithmetic (the
paper's precision for the operator inside CG, Sec. 5.1).

metric value = (applies in the solve) x n_dofs / (solve time): the FP64 SIPG
operator applies in DoF/s sustained over the whole solve (CG vector updates and
reductions included); ms_per_step is the time to the 1e-10 solve.  Nothing in
the timed solves is instrumented; the per-apply time of the roofline comes from
one instrumented solve after them.  The same solve with the operator in
double-float arithmetic, with the FP32 multigrid preconditioner, and the FP32
operator are reported as extra keys.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 it runs under torchrun, one independent replica of the workload per
GPU (the path has no data exchange on one mesh per GPU: "replicas only").
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DoF/s of SIPG operator apply (FP64, FP32) and % HBM roofline; time to 1e-10 Poisson solve"
UNIT = "DoF/s"
WORKLOAD = dict(n=(32, 32, 32), lo=(0.0, -1.0, 0.0), hi=(2 * math.pi, 1.0, math.pi),
                bc_lo=("periodic", "dirichlet", "periodic"), bc_hi=("periodic", "dirichlet", "periodic"),
                mapping="channel", gamma=1.8, k=4)
RTOL = 1e-10
CHECK_EVERY = 16


def fma_per_dof(p):
    """FMAs per DoF of one Laplace apply in the Kronecker-sum evaluation (interior
    faces): three line operators (p^2 + 6p per line: 1D stiffness, two faces with
    own and neighbour normal derivative and the derivative scatter), five 1D mass
    contractions (p^2 each) -> 8p + 18 per DoF."""
    return 8 * p + 18


# FP32 flops of one double-float operation (dfloat.cuh): fma = 1 FMUL + 3 FFMA
# (exact product error) + TwoSum (6 FADD) + 2 FADD + renormalisation (3 FADD);
# add = TwoSum + 2 + 3; FFMA counts 2 flops.
DF_FMA_FLOPS = 1 + 3 * 2 + 6 + 2 + 3
DF_ADD_FLOPS = 6 + 2 + 3


def df_ops_per_dof(p, dots=True):
    """Double-float operations per DoF of one uniform-viscosity apply (interior
    faces), counted from the kernel: per thread (one line in each of the phases
    X, Y, Z) three line operators with P^2 + 4P + 2 fma and 4 adds, five 1D mass
    contractions (5 P^2 fma), P + P adds in Y2/X2, 9 adds of penalty values, and
    with dots P fma + 2P adds.  A thread covers P DoFs."""
    fma = 3 * (p * p + 4 * p + 2) + 5 * p * p + (p if dots else 0)
    add = 3 * 4 + 2 * p + 9 + (2 * p if dots else 0)
    return fma / p, add / p


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
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
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sms) if sms else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sms)}


def aggregate_replicas(t_local, units_local, dist=None):
    """Whole-job throughput of independent replicas: the units of all ranks
    over the slowest rank's time (max over ranks).  Returns (value, t_max)."""
    import torch
    world = dist.get_world_size() if dist is not None and dist.is_initialized() else 1
    if world > 1:
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(t_local)], device=dev, dtype=torch.float64)
        u = torch.tensor([float(units_local)], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        return u.item() / t.item(), t.item()
    return units_local / t_local, t_local


def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != n_gpus and world > 1:
        raise SystemExit("WORLD_SIZE %d != --gpus %d" % (world, n_gpus))
    return rank, world, local


def manufactured_f(X):
    """f = -Laplace(u) for u = sin x cos(pi y/2) sin 2z, at the given points (n, 3)."""
    import numpy as np
    return (5 + math.pi ** 2 / 4) * np.sin(X[:, 0]) * np.cos(math.pi * X[:, 1] / 2) * np.sin(2 * X[:, 2])


BENCH_CONFIG = {"workload": "poisson_channel_32x32x32_k4_jacobi_pcg_1e-10", "dofs": 4096000, "k": 4,
                "gamma": 1.8, "rtol": RTOL, "cuda_graph_chunk": CHECK_EVERY, "f64_arithmetic": "native",
                "l2": "256 MB buffer written between timed steps (outside the timed events)"}


def bench_config(world=1):
    """The config dict of both arms (identical keys and values)."""
    return dict(BENCH_CONFIG, parallelism="replicas" if world > 1 else "single")


# The oracle timings of the five configurations: mesh, degree, components,
# operator coefficients and the sampled fraction of the cells (about a second
# of single-core oracle work per sampled apply).
_CH = dict(lo=(0.0, -1.0, 0.0), hi=(2 * math.pi, 1.0, math.pi), mapping="channel", gamma=1.8)
ORACLE_CONFIGS = {
    "c1": dict(n=(4, 4, 4), lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), bc=("periodic",) * 3, mapping="affine",
               gamma=1.8, k=3, ncomp=1, frac=1.0, kw={}, label="4^3 periodic cube, k=3, Laplace"),
    "c2": dict(WORKLOAD, bc=None, ncomp=1, frac=1.0 / 16, kw={}, label="32^3 k=4 channel Poisson operator"),
    "c3": dict(_CH, n=(64, 64, 64), bc=("periodic", "dirichlet", "periodic"), k=3, ncomp=3, frac=1.0 / 256,
               kw=dict(mass_coef=1500.0, nu=1 / 180), label="64^3 k=3 channel Helmholtz, 3 components"),
    "c4": dict(_CH, n=(48, 48, 48), bc=("periodic", "neumann", "periodic"), k=5, ncomp=1, frac=1.0 / 128, kw={},
               label="48^3 k=5 Neumann channel Laplacian"),
    "c5": dict(_CH, n=(32, 32, 32), bc=("periodic", "dirichlet", "periodic"), k=3, ncomp=1, frac=1.0 / 32,
               kw=dict(mass_coef=1500.0, nu_cell="lognormal"), label="32^3 k=3 channel Helmholtz, per-cell nu"),
}

_ORACLE = {}


def _oracle_state(frac, cfg="c2"):
    """The oracle operator of a configuration, its seeded cell sample and an
    input (cached per process)."""
    key = (cfg, frac)
    if key not in _ORACLE:
        import numpy as np
        from oracle.mesh import MeshSpec
        from oracle.sipg import SIPG
        from paper_1607_01323_gb300 import inputs
        c = ORACLE_CONFIGS[cfg]
        bc_lo = c["bc"] if c["bc"] else c["bc_lo"]
        bc_hi = c["bc"] if c["bc"] else c["bc_hi"]
        spec = MeshSpec(*c["n"], lo=c["lo"], hi=c["hi"], bc_lo=bc_lo, bc_hi=bc_hi, mapping=c["mapping"],
                        gamma=c["gamma"])
        t0 = time.time()
        op = SIPG(spec, c["k"])
        setup = time.time() - t0
        ncell = spec.ncell
        if frac >= 1.0:
            cells = np.arange(ncell)
        else:
            pick = inputs.u64(0, "oracle_sample", 0, int(ncell * frac)) % np.uint64(ncell)
            cells = np.unique(pick.astype(np.int64))
        if cfg == "c2":
            X = op.node_coordinates().reshape(-1, 3)
            x = manufactured_f(X)
        else:
            x = inputs.uniform(0, "x", c["ncomp"] * ncell * op.P).reshape(c["ncomp"], -1)
        kw = dict(c["kw"])
        if kw.get("nu_cell") == "lognormal":
            kw["nu_cell"] = np.exp(0.5 * inputs.normal(0, "xi", ncell)) / 180.0
        _ORACLE[key] = dict(op=op, cells=cells, x=x, kw=kw, setup=setup, ncell=ncell)
    return _ORACLE[key]


def _oracle_apply_part(frac, part, nparts, cfg="c2"):
    """One oracle apply restricted to the part-th of nparts slices of the sampled
    cells (a process-pool task); returns the process CPU seconds it used."""
    import numpy as np
    st = _oracle_state(frac, cfg)
    mask = np.zeros(st["ncell"], dtype=bool)
    mask[st["cells"][part::nparts]] = True
    c0 = time.process_time()
    st["op"].apply(st["x"], targets=mask, **st["kw"])
    return time.process_time() - c0


class OracleSample:
    """The oracle as it stands (dense-quadrature element-by-element FP64 apply)
    on one of the configurations (default: the bench's 32^3 k=4 channel
    problem), bounded: each timed unit is one operator apply restricted to a
    fixed seeded sample of ``frac`` of the cells, counted as (sampled DoFs) per
    second, i.e. the same DoF/s of operator apply.  With workers > 1 the
    sample is split over that many spawned processes (one per host core); the
    oracle's CG adds only vector operations around its applies."""

    def __init__(self, frac=1.0 / 16, workers=1, cfg="c2"):
        self.frac, self.workers, self.cfg = frac, workers, cfg
        self.pool = None
        if workers > 1:
            import multiprocessing as mp
            from concurrent.futures import ProcessPoolExecutor
            # spawned (not forked) workers, one BLAS thread each
            saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
            for k in saved:
                os.environ[k] = "1"
            try:
                self.pool = ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))
                t0 = time.time()
                list(self.pool.map(_oracle_state, [frac] * workers, [cfg] * workers))
                self.setup = time.time() - t0
            finally:
                for k, v in saved.items():
                    if v is None:
                        os.environ.pop(k, None)
                    else:
                        os.environ[k] = v
            st = _oracle_state_meta(frac, cfg)
        else:
            st = _oracle_state(frac, cfg)
            self.setup = st["setup"]
        c = ORACLE_CONFIGS[cfg]
        self.ncells, self.ncell = len(st["cells"]), st["ncell"]
        self.sample_dofs = self.ncells * (c["k"] + 1) ** 3 * c["ncomp"]

    def step(self):
        """(wall seconds, CPU seconds) of one sampled apply."""
        t0 = time.time()
        if self.pool is None:
            cpu = _oracle_apply_part(self.frac, 0, 1, self.cfg)
        else:
            n = self.workers
            cpu = sum(self.pool.map(_oracle_apply_part, [self.frac] * n, range(n), [n] * n, [self.cfg] * n))
        return time.time() - t0, cpu

    def close(self):
        if self.pool is not None:
            self.pool.shutdown()
            self.pool = None

    def describe(self, n, wall):
        return ("%d oracle FP64 applies restricted to a seeded sample of %d of %d cells (%d DoF each) of the "
                "%s on %d process(es), %.1f s wall after %.1f s oracle setup; sampled DoF per second"
                % (n, self.ncells, self.ncell, self.sample_dofs, ORACLE_CONFIGS[self.cfg]["label"], self.workers,
                   wall, self.setup))


def _oracle_state_meta(frac, cfg="c2"):
    """The sampled cells of a configuration without building the operator."""
    import numpy as np
    from paper_1607_01323_gb300 import inputs
    n = ORACLE_CONFIGS[cfg]["n"]
    ncell = n[0] * n[1] * n[2]
    if frac >= 1.0:
        return dict(cells=np.arange(ncell), ncell=ncell)
    pick = inputs.u64(0, "oracle_sample", 0, int(ncell * frac)) % np.uint64(ncell)
    return dict(cells=np.unique(pick.astype(np.int64)), ncell=ncell)


def time_oracle(workers, max_seconds, frac=None, warmup=1, steps=None, cfg="c2"):
    """Sampled oracle applies on `workers` processes: the DoF/s and its record."""
    s = OracleSample(ORACLE_CONFIGS[cfg]["frac"] if frac is None else frac, workers, cfg)
    try:
        for _ in range(warmup):
            s.step()
        walls, cpus = [], []
        while (steps is None and sum(walls) < max_seconds and len(walls) < 64) or (steps is not None and
                                                                                 len(walls) < steps):
            w, c = s.step()
            walls.append(w)
            cpus.append(c)
        value = len(walls) * s.sample_dofs / sum(walls)
        rec = {"value": value, "unit": UNIT, "cores": max(1, round(sum(cpus) / sum(walls))), "kind": "oracle",
               "sample": s.describe(len(walls), sum(walls)), "host_cpus": os.cpu_count()}
        return value, rec, sum(walls)
    finally:
        s.close()


def cpu_baseline(max_seconds=12.0):
    """The oracle on all host cores (the reported baseline) and on one core."""
    ncpu = os.cpu_count() or 1
    _, allc, _ = time_oracle(ncpu, max_seconds)
    _, one, _ = time_oracle(1, max_seconds)
    allc["single_core"] = {k: one[k] for k in ("value", "cores", "sample")}
    return allc


def run_reference(args):
    rank, world, _ = dist_setup(args.gpus)
    if rank != 0:
        return
    ncpu = os.cpu_count() or 1
    value, rec, wall = time_oracle(ncpu, None, warmup=args.warmup, steps=args.steps)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": bench_config(world), "cpu_baseline": rec,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_1607_01323_gb300 import Mesh, apply_laplace_f32, apply_laplace_f64, apply_mass_f64, cg_solve

    w = WORKLOAD
    m = Mesh(w["n"], w["lo"], w["hi"], w["bc_lo"], w["bc_hi"], mapping=w["mapping"], gamma=w["gamma"], k=w["k"])
    m.set_f64_arithmetic(args.f64)
    N = m.n_dofs
    p = w["k"] + 1
    X = m.node_coordinates()
    b = apply_mass_f64(m, torch.tensor(manufactured_f(X), device="cuda"))
    x = torch.zeros_like(b)
    flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2
    opts = dict(precond="jacobi", rtol=RTOL, use_graph=1, check_every=CHECK_EVERY)

    def solve(mesh):
        x.zero_()
        return cg_solve(mesh, b, x, **opts)[1]

    for _ in range(args.warmup):
        res = solve(m)
    torch.cuda.synchronize()
    # the timed steps: whole solves, nothing instrumented
    m.profile_read(reset=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    iters = []
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record()
        res = solve(m)
        ev[i][1].record()
        iters.append(res.iters)
        if not res.converged:
            raise SystemExit("solve did not converge: %r" % res)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    _, _, launches = m.profile_read(reset=True)
    t_steps = [a.elapsed_time(bb) for a, bb in ev]
    n_applies = sum(it + 1 for it in iters)  # initial residual + one per iteration
    value, t_total = aggregate_replicas(sum(t_steps) / 1e3, n_applies * N, dist if world > 1 else None)
    ms_per_step = 1e3 * t_total / args.steps

    def apply_in_solve(mesh):
        """Average duration of the operator launches inside one solve of the same
        kind (CUDA events around each apply on the solve's stream), taken in an
        instrumented solve after the timed steps."""
        mesh.profile_enable(True)
        mesh.profile_read(reset=True)
        flush.fill_(0.5)
        solve(mesh)
        torch.cuda.synchronize()
        ms, n, _ = mesh.profile_read(reset=True)
        mesh.profile_enable(False)
        return ms / max(n, 1), n

    def apply_isolated(mesh, fn, xin, reps=20):
        """Average duration of single applies, L2 flushed before each."""
        yout = torch.empty_like(xin)
        for _ in range(3):
            fn(mesh, xin, yout)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for i in range(reps):
            flush.fill_(float(i))
            e0.record()
            fn(mesh, xin, yout)
            e1.record()
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / reps

    avg_apply_ms, timed_applies = apply_in_solve(m)
    iso_apply_ms = apply_isolated(m, apply_laplace_f64, b)

    # accuracy of the last solve: || u_h - I u ||_M against the nodal interpolant
    # of the exact solution u = sin x cos(pi y/2) sin 2z (a diagnostic, outside
    # the timed region)
    u_ex = torch.tensor(np.sin(X[:, 0]) * np.cos(math.pi * X[:, 1] / 2) * np.sin(2 * X[:, 2]), device="cuda")
    solve(m)
    err = x - u_ex
    l2_err = math.sqrt(max(torch.dot(err, apply_mass_f64(m, err)).item(), 0.0))
    l2_u = math.sqrt(torch.dot(u_ex, apply_mass_f64(m, u_ex)).item())

    # end to end through the public API: pinned host rhs -> device, solve, solution -> host
    hb = torch.empty(N, dtype=torch.float64, pin_memory=True)
    hb.copy_(b.cpu())
    hx = torch.empty(N, dtype=torch.float64, pin_memory=True)
    db = torch.empty_like(b)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_iters = 0
    torch.cuda.synchronize()
    e2e_ms = 0.0
    for i in range(args.steps):
        flush.fill_(float(i))
        e0.record()
        db.copy_(hb, non_blocking=True)
        x.zero_()
        _, r2 = cg_solve(m, db, x, **opts)
        hx.copy_(x, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        e2e_ms += e0.elapsed_time(e1)
        e2e_iters += r2.iters + 1
    e2e_value = world * e2e_iters * N / (e2e_ms / 1e3)

    def timed_solves(mesh, o, reps):
        """Average ms and the iterations of `reps` solves of b (L2 flushed)."""
        for _ in range(2):
            x.zero_()
            cg_solve(mesh, b, x, **o)
        torch.cuda.synchronize()
        ms, it = [], 0
        for i in range(reps):
            flush.fill_(float(i))
            x.zero_()
            e0.record()
            _, rr = cg_solve(mesh, b, x, **o)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            it = rr.iters
            if not rr.converged:
                raise SystemExit("solve did not converge: %r" % rr)
        return sum(ms) / len(ms), it

    # the same Jacobi-PCG with the FP64 operator evaluated in double-float
    # (FP32 pairs, 48 bits, a power-of-two scale per call) on the FP32 pipes
    mdf = Mesh(w["n"], w["lo"], w["hi"], w["bc_lo"], w["bc_hi"], mapping=w["mapping"], gamma=w["gamma"], k=w["k"])
    mdf.set_f64_arithmetic("double_float")
    df_ms, df_iters = timed_solves(mdf, opts, max(3, min(args.steps, 10)))
    df_apply_ms, _ = apply_in_solve(mdf)
    df_iso_ms = apply_isolated(mdf, apply_laplace_f64, b)
    del mdf

    # the same solve with the multigrid preconditioner of Sec. 5.1 (outside the
    # timed steps; its set-up -- level tables, diagonals, Lanczos estimates, the
    # dense coarse operator -- is built once and cached on the mesh)
    from paper_1607_01323_gb300 import mg_setup
    mg_opts = dict(precond="gmg_f32", rtol=RTOL, use_graph=1, check_every=CHECK_EVERY)
    torch.cuda.synchronize()
    t_setup = time.perf_counter()
    mg_info = mg_setup(m, precond="gmg_f32")
    mg_setup_ms = 1e3 * (time.perf_counter() - t_setup)
    mg_ms, mg_iters = timed_solves(m, mg_opts, max(3, min(args.steps, 10)))

    # FP32 operator apply throughput on the same mesh (outside the timed step)
    f32_ms = apply_isolated(m, apply_laplace_f32, b.float())

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs")
    bytes_apply = 16.0 * N  # algorithmic: read x, write y (FP64); geometry is O(layers)
    achieved_gbs = bytes_apply / (avg_apply_ms / 1e3) / 1e9
    # the FP64 pipe: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz
    flops_per_dof = 2.0 * fma_per_dof(p)
    fp64_peak = 152 * 2 * 2 * 2.07e9 / 1e12
    fp64_tflops = flops_per_dof * N / (avg_apply_ms / 1e3) / 1e12
    # double-float: FP32 operations of the kernel against the FP32 pipes
    fma_d, add_d = df_ops_per_dof(p, dots=True)
    df_flops = fma_d * DF_FMA_FLOPS + add_d * DF_ADD_FLOPS
    fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12
    traffic = None
    tf = os.path.join(ROOT, "profiles", "traffic_apply_uniform_f64_channel32_k4.json")
    if os.path.exists(tf):
        with open(tf) as f:
            traffic = json.load(f).get("dram_bytes_per_launch")
    bound_dofs = min(hbm * 1e9 / 16.0 if hbm else float("inf"), fp64_peak * 1e12 / flops_per_dof)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.f64 == "native" else "f32x2",
        "data": "synthetic",
        "config": dict(bench_config(world), f64_arithmetic=args.f64),
        "cg_iters": iters[-1],
        "time_to_solve_s": ms_per_step / 1e3,
        "solution_error": {"l2_vs_nodal_interpolant": l2_err, "relative": l2_err / l2_u,
                           "note": "|| u_h - I u ||_M of the manufactured solution after the timed solves"},
        "apply_f64": {"avg_ms_in_solve": avg_apply_ms, "avg_ms_isolated": iso_apply_ms,
                      "dofs_per_s": N / (avg_apply_ms / 1e3), "timed_launches": timed_applies,
                      "hbm_frac": achieved_gbs / hbm if hbm else None,
                      "note": "operator launches of one instrumented solve after the timed steps (events on the "
                              "solve's stream); isolated: single applies, L2 flushed before each"},
        "roofline": {"bound": "hbm", "kernel": "apply_uniform_kernel<double,double,5>", "achieved": achieved_gbs,
                     "peak": hbm, "unit": "GB/s", "frac": achieved_gbs / hbm if hbm else None,
                     "traffic": traffic, "bytes_per_dof": 16,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy), of measured",
                     "alu": {"bound": "fp64 pipe", "achieved": fp64_tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                             "frac": fp64_tflops / fp64_peak, "flops_per_dof": flops_per_dof,
                             "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk/SM x 2 x 2.07 GHz"},
                     "bound_dofs_per_s": bound_dofs,
                     "apply_frac_of_bound": (N / (avg_apply_ms / 1e3)) / bound_dofs},
        "double_float": {
            "solve_ms": df_ms, "cg_iters": df_iters, "apply_avg_ms_in_solve": df_apply_ms,
            "apply_avg_ms_isolated": df_iso_ms, "dofs_per_s": N / (df_apply_ms / 1e3),
            "hbm_frac": (bytes_apply / (df_apply_ms / 1e3) / 1e9) / hbm if hbm else None,
            "fp32_pipe_utilisation": df_flops * N / (df_apply_ms / 1e3) / 1e12 / fp32_peak,
            "note": "FP64 data, operator in FP32 pairs (~2^-46 per operation, exponent range of FP64 through a "
                    "power-of-two scale per call); parity 1e-12 ||A|| ||x|| as native (tests); pipe utilisation "
                    "counts the FP32 operations of the emulation against 152 x 128 x 2 x 2.07 GHz"},
        "apply_f32": {"avg_ms": f32_ms, "dofs_per_s": N / (f32_ms / 1e3),
                      "hbm_frac": (8.0 * N / (f32_ms / 1e3) / 1e9) / hbm if hbm else None,
                      "note": "separate timing of the FP32 operator on the same mesh, L2 flushed per launch"},
        "gmg_solve": {"ms": mg_ms, "cg_iters": mg_iters, "setup_ms": mg_setup_ms,
                      "levels": mg_info["n_cells"], "coarse_degree": mg_info["coarse_degree"],
                      "speedup_vs_jacobi": ms_per_step / mg_ms,
                      "note": "CG with one FP32 geometric-multigrid V-cycle per iteration (Chebyshev degree 5, "
                              "range 20), same rhs and tolerance; set-up cached and not timed"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 8 * N},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def run_apply_only(args):
    """A few operator applies on the bench mesh (or --cells/--k), for ncu captures."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1607_01323_gb300 import Mesh, apply_laplace_f32, apply_laplace_f64
    w = dict(WORKLOAD)
    n = (args.cells,) * 3 if args.cells else w["n"]
    k = args.k if args.k else w["k"]
    m = Mesh(n, w["lo"], w["hi"], w["bc_lo"], w["bc_hi"], mapping=w["mapping"], gamma=w["gamma"], k=k)
    m.set_f64_arithmetic(args.f64)
    dt = torch.float64 if args.precision == "f64" else torch.float32
    x = torch.rand(m.n_dofs, dtype=dt, device="cuda")
    y = torch.empty_like(x)
    f = apply_laplace_f64 if args.precision == "f64" else apply_laplace_f32
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for i in range(args.reps):
        ev[0].record()
        f(m, x, y)
        ev[1].record()
        torch.cuda.synchronize()
        print("apply %s n=%s k=%d dofs=%d: %.4f ms" % (args.precision, n, k, m.n_dofs, ev[0].elapsed_time(ev[1])))


def run_solve_only(args):
    """A few Jacobi-PCG solves of the bench problem (native or double-float FP64
    operator, or --precond), timed with CUDA events; for ncu launch lists."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1607_01323_gb300 import Mesh, apply_mass_f64, cg_solve
    w = dict(WORKLOAD)
    n = (args.cells,) * 3 if args.cells else w["n"]
    k = args.k if args.k else w["k"]
    m = Mesh(n, w["lo"], w["hi"], w["bc_lo"], w["bc_hi"], mapping=w["mapping"], gamma=w["gamma"], k=k)
    m.set_f64_arithmetic(args.f64)
    b = apply_mass_f64(m, torch.tensor(manufactured_f(m.node_coordinates()), device="cuda"))
    x = torch.zeros_like(b)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for i in range(args.reps):
        x.zero_()
        ev[0].record()
        _, r = cg_solve(m, b, x, precond=args.precond, rtol=RTOL, use_graph=1, check_every=CHECK_EVERY)
        ev[1].record()
        torch.cuda.synchronize()
        print("solve %s %s n=%s k=%d dofs=%d: %d iterations, %.3f ms" % (args.f64, args.precond, n, k, m.n_dofs,
                                                                          r.iters, ev[0].elapsed_time(ev[1])))


def run_convective_only(args):
    """A few convective-term applies on the bench channel (or --cells/--k)
    with a laminar profile plus noise, timed with CUDA events; for ncu captures."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1607_01323_gb300 import Mesh, apply_convective_f64, inputs
    w = dict(WORKLOAD)
    n = (args.cells,) * 3 if args.cells else w["n"]
    k = args.k if args.k else w["k"]
    m = Mesh(n, w["lo"], w["hi"], w["bc_lo"], w["bc_hi"], mapping=w["mapping"], gamma=w["gamma"], k=k)
    m.set_f64_arithmetic(args.f64)
    N = m.n_dofs
    X = m.node_coordinates()
    u = torch.tensor(np.concatenate([(1 - X[:, 1] ** 2) + 0.1 * inputs.normal(0, "ux", N),
                                     0.1 * inputs.normal(0, "uy", N), 0.1 * inputs.normal(0, "uz", N)]),
                     device="cuda")
    y = torch.empty_like(u)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for i in range(args.reps):
        ev[0].record()
        apply_convective_f64(m, u, y=y)
        ev[1].record()
        torch.cuda.synchronize()
        print("convective %s n=%s k=%d dofs=%d: %.4f ms" % (args.f64, n, k, 3 * N, ev[0].elapsed_time(ev[1])))


def run_vcycle_only(args):
    """Multigrid set-up and a few V-cycles on the bench mesh (or --cells/--k),
    timed with CUDA events; for ncu launch lists of the V-cycle."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1607_01323_gb300 import Mesh, mg_setup, mg_vcycle
    w = dict(WORKLOAD)
    n = (args.cells,) * 3 if args.cells else w["n"]
    k = args.k if args.k else w["k"]
    m = Mesh(n, w["lo"], w["hi"], w["bc_lo"], w["bc_hi"], mapping=w["mapping"], gamma=w["gamma"], k=k)
    info = mg_setup(m, precond="gmg_f32")
    r = torch.rand(m.n_dofs, dtype=torch.float64, device="cuda")
    z = torch.empty_like(r)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for i in range(args.reps):
        ev[0].record()
        mg_vcycle(m, r, z)
        ev[1].record()
        torch.cuda.synchronize()
        print("vcycle n=%s k=%d dofs=%d levels=%d coarse_degree=%d: %.4f ms" % (
            n, k, m.n_dofs, info["nlevels"], info["coarse_degree"], ev[0].elapsed_time(ev[1])))


def _timed(fn, reps=3):
    """Median wall time (s) of fn() bracketed by device synchronisation."""
    import torch
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    return statistics.median(ts), out


def run_oracle_timings(args):
    """The oracle (as it stands) on the GPU host's cores, every configuration:
    the sampled FP64 apply on all cores (one spawned process per core) and on
    one core; the oracle's Jacobi-PCG solve to 1e-10 for the 4^3 cube
    (assembled CSR, one core) and, for the bench's 32^3 k=4 problem, the time
    of one full all-core apply times the GPU solve's 342 iterations (the
    oracle's CG adds only vector operations around its applies)."""
    import numpy as np
    ncpu = os.cpu_count() or 1
    out = {"workload": "oracle", "host_cpus": ncpu, "applies": {}}
    for cfg in ("c1", "c2", "c3", "c4", "c5"):
        va, ra, _ = time_oracle(ncpu, args.oracle_seconds, cfg=cfg)
        v1, r1, _ = time_oracle(1, args.oracle_seconds, cfg=cfg)
        out["applies"][cfg] = {"all_cores_dofs_per_s": va, "one_core_dofs_per_s": v1, "cores_used": ra["cores"],
                               "sample_all_cores": ra["sample"], "sample_one_core": r1["sample"]}
    # oracle Jacobi-PCG on the 4^3 periodic cube, k = 3 (zero-mean rhs)
    from oracle import solvers
    st = _oracle_state(1.0, "c1")
    A = st["op"].assemble()
    b = st["x"][0] - st["x"][0].mean()
    t0 = time.time()
    xs, it, rel = solvers.cg(lambda v: A @ v, b, rtol=1e-10, zero_mean=True, precond=lambda r: r / A.diagonal())
    out["cg_c1"] = {"seconds": time.time() - t0, "iters": it, "relres": rel, "cores": 1,
                    "note": "assembled CSR (4096 unknowns), Jacobi-PCG to 1e-10, zero-mean rhs"}
    # the bench problem: one full apply on all cores, times the GPU solve's iterations
    va, ra, wall = time_oracle(ncpu, None, frac=1.0, warmup=0, steps=1, cfg="c2")
    t_apply = 4096000 / va
    out["cg_c2_estimate"] = {"seconds_per_apply_all_cores": t_apply, "iters": 342,
                             "estimated_solve_s": 343 * t_apply, "sample": ra["sample"],
                             "note": "one full oracle apply of the 32^3 k=4 Poisson operator on all cores times "
                                     "the 343 applies of the 1e-10 Jacobi-PCG solve (the GPU's iteration count)"}
    print(json.dumps(out))


def run_config(args):
    """Timings of the other workload configurations (one JSON line each):
    c1: the 4^3 periodic unit cube at k=3 (operator apply only);
    c3: 3-component viscous Helmholtz on the 64^3 k=3 channel (apply, autotune,
        graph-captured CG with M^-1 and Jacobi), in the Laplace form of the
        configuration and in the paper's divergence form (coupled components),
        and the convective term of the explicit step on the same velocity;
    c4: Neumann-channel Poisson 48^3 k=5, FP32 Chebyshev(4) + FP64 flexible CG
        versus plain FP64 Jacobi CG;
    c5: adjoint gradient on the 32^3 k=3 channel with per-cell viscosity;
    v3c: divergence, gradient, tau_D and the div-div local projection of the
        pressure-projection step on the 32^3 k=4 channel;
    ns: the dual-splitting time step (BDF3, V3c) on the 32^3 k=4 channel;
    perturbed: the general-metric FP64 apply on a 32^3 perturbed box, k=4;
    mg_scaling: multigrid and Jacobi PCG iteration counts on refined channels."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1607_01323_gb300 import (Mesh, apply_helmholtz_f64, apply_laplace_f32, apply_laplace_f64,
                                        apply_mass_f64, autotune, cg_solve, inputs)
    w = WORKLOAD
    out = {"workload": args.workload, "f64_arithmetic": args.f64}
    if args.workload == "c1":
        m = Mesh((4, 4, 4), k=3)  # periodic unit cube, affine, tau = 192
        m.set_f64_arithmetic(args.f64)
        x = torch.tensor(inputs.uniform(0, "x", m.n_dofs), device="cuda")
        y = torch.empty_like(x)
        t, _ = _timed(lambda: [apply_laplace_f64(m, x, y) for _ in range(100)], reps=5)
        out["apply_f64"] = {"us": 1e6 * t / 100, "dofs": m.n_dofs, "note": "launch-latency bound (64 cells)"}
    elif args.workload == "c3":
        m = Mesh((64, 64, 64), w["lo"], w["hi"], w["bc_lo"], w["bc_hi"], mapping="channel", gamma=1.8, k=3)
        m.set_f64_arithmetic(args.f64)
        N = m.n_dofs
        cm, nu = 1.5 / 1e-3, 1 / 180
        X = m.node_coordinates()
        u_in = np.concatenate([(1 - X[:, 1] ** 2) + 0.1 * inputs.normal(0, "ux", N),
                               0.1 * inputs.normal(0, "uy", N), 0.1 * inputs.normal(0, "uz", N)])
        u = torch.tensor(u_in, device="cuda")
        y = torch.empty_like(u)
        out["cpb_default"] = m.cells_per_block(0)
        t_def, _ = _timed(lambda: apply_helmholtz_f64(m, u, cm, nu, y=y), reps=5)
        out["cpb_autotuned"] = autotune(m, 0)
        t_apply, _ = _timed(lambda: apply_helmholtz_f64(m, u, cm, nu, y=y), reps=5)
        out["apply_f64"] = {"ms_default_cpb": 1e3 * t_def, "ms": 1e3 * t_apply, "dofs": 3 * N,
                            "dofs_per_s": 3 * N / t_apply}
        rhs = cm * apply_mass_f64(m, u)
        for pc in ("invmass", "jacobi"):
            x = torch.zeros_like(rhs)
            for graph in (1, 0):
                t, (x, res) = _timed(lambda: cg_solve(m, rhs, torch.zeros_like(rhs), op="helmholtz",
                                                      mass_coef=cm, nu=nu, precond=pc, rtol=1e-10,
                                                      use_graph=graph), reps=3)
                out["solve_%s_%s" % (pc, "graph" if graph else "loop")] = {
                    "s": t, "iters": res.iters, "relres": res.relres,
                    "dof_applies_per_s": 3 * N * (res.iters + 1) / t}
        # the paper's divergence-form viscous operator (eps(u), coupled
        # components) on the same mesh and input, and its M^-1-preconditioned CG
        from paper_1607_01323_gb300 import apply_viscous_f64
        t_v, _ = _timed(lambda: apply_viscous_f64(m, u, cm, nu, y=y), reps=5)
        out["apply_viscous_div_form"] = {"ms": 1e3 * t_v, "dofs": 3 * N, "dofs_per_s": 3 * N / t_v}
        t, (x, res) = _timed(lambda: cg_solve(m, rhs, torch.zeros_like(rhs), op="viscous", mass_coef=cm, nu=nu,
                                              precond="invmass", rtol=1e-10), reps=3)
        out["solve_viscous_div_form_invmass_graph"] = {"s": t, "iters": res.iters, "relres": res.relres,
                                                       "dof_applies_per_s": 3 * N * (res.iters + 1) / t}
        # the convective term of the explicit step (LLF flux, floor(3k/2)+1
        # Gauss points) on the same mesh and velocity
        from paper_1607_01323_gb300 import apply_convective_f64
        cpb_c = m.cells_per_block(2)
        t_c0, _ = _timed(lambda: apply_convective_f64(m, u, y=y), reps=5)
        cpb_ct = autotune(m, 2)
        t_c, _ = _timed(lambda: apply_convective_f64(m, u, y=y), reps=5)
        out["apply_convective_llf"] = {"ms_default_cpb": 1e3 * t_c0, "cpb_default": cpb_c, "cpb_autotuned": cpb_ct,
                                       "ms": 1e3 * t_c, "dofs": 3 * N, "dofs_per_s": 3 * N / t_c,
                                       "quadrature_points_per_dir": (3 * 3) // 2 + 1}
    elif args.workload == "c4":
        m = Mesh((48, 48, 48), w["lo"], w["hi"], ("periodic", "neumann", "periodic"),
                 ("periodic", "neumann", "periodic"), mapping="channel", gamma=1.8, k=5)
        m.set_f64_arithmetic(args.f64)
        N = m.n_dofs
        b = inputs.uniform(0, "b", N)
        b -= b.mean()
        bt = torch.tensor(b, device="cuda")
        x32 = bt.float()
        y32 = torch.empty_like(x32)
        y64 = torch.empty_like(bt)
        t32, _ = _timed(lambda: apply_laplace_f32(m, x32, y32), reps=5)
        t64, _ = _timed(lambda: apply_laplace_f64(m, bt, y64), reps=5)
        out["apply_f32"] = {"ms": 1e3 * t32, "dofs_per_s": N / t32}
        out["apply_f64"] = {"ms": 1e3 * t64, "dofs_per_s": N / t64}
        tc, (xc, rc) = _timed(lambda: cg_solve(m, bt, precond="cheb_f32", cheb_degree=4, zero_mean=1,
                                                rtol=1e-10), reps=2)
        tj, (xj, rj) = _timed(lambda: cg_solve(m, bt, precond="jacobi", zero_mean=1, rtol=1e-10), reps=2)
        d = (xc - xc.mean()) - (xj - xj.mean())
        out["mixed_cheb4_fcg"] = {"s": tc, "iters": rc.iters, "relres": rc.relres}
        out["plain_f64_jacobi_cg"] = {"s": tj, "iters": rj.iters, "relres": rj.relres}
        out["speedup"] = tj / tc
        out["rel_diff_solutions"] = (torch.linalg.norm(d) / torch.linalg.norm(xj - xj.mean())).item()
    elif args.workload == "c5":
        from paper_1607_01323_gb300.autograd import helmholtz_solve, mass_norm_loss
        m = Mesh((32, 32, 32), w["lo"], w["hi"], w["bc_lo"], w["bc_hi"], mapping="channel", gamma=1.8, k=3)
        cm = 1500.0
        nu = torch.tensor(np.exp(0.5 * inputs.normal(0, "xi", m.ncell)) / 180.0, device="cuda")
        X = m.node_coordinates()
        fc = np.sin(X[:, 0]) * np.cos(math.pi * X[:, 1] / 2) * np.sin(2 * X[:, 2])
        ph = 2 * math.pi * (0.5 * (inputs.uniform(0, "phase", 2) + 1))
        ut = torch.tensor(np.cos(math.pi * X[:, 1] / 2) * (1 + 0.5 * np.sin(X[:, 0] + ph[0]) *
                                                           np.cos(X[:, 2] + ph[1])), device="cuda")
        f = apply_mass_f64(m, torch.tensor(fc, device="cuda"))

        def fwd():
            return mass_norm_loss(m, helmholtz_solve(m, nu, f, cm, rtol=1e-10), ut)

        def fwd_bwd():
            nu_t = nu.clone().requires_grad_(True)
            J = mass_norm_loss(m, helmholtz_solve(m, nu_t, f, cm, rtol=1e-10), ut)
            J.backward()
            return nu_t.grad

        t_f, _ = _timed(fwd, reps=3)
        t_fb, g = _timed(fwd_bwd, reps=3)
        out["forward_s"] = t_f
        out["forward_backward_s"] = t_fb
        out["backward_over_forward"] = (t_fb - t_f) / t_f
        out["finite_difference_estimate_s"] = 2 * m.ncell * t_f
        out["grad_norm"] = torch.linalg.norm(g).item()
    elif args.workload == "ns":
        # the dual-splitting step on the bench channel: laminar profile plus
        # noise, body force 2 nu, BDF3, div-div penalty, GMG pressure solve;
        # relative tolerances 1e-6 with extrapolated initial guesses (Sec. 5.1)
        from paper_1607_01323_gb300 import NavierStokes
        nu, dt = 1 / 180, 1e-3
        n_ns = (args.cells,) * 3 if args.cells else w["n"]
        ns = NavierStokes(n_ns, w["lo"], w["hi"], w["bc_lo"], w["bc_hi"], mapping=w["mapping"], gamma=w["gamma"],
                          k=w["k"], nu=nu, dt=dt, order=3, zeta=1.0, pressure_precond="gmg_f32", rtol_pressure=1e-6,
                          rtol_viscous=1e-6, rtol_projection=1e-8, f64_arithmetic=args.f64)
        N = ns.n_dofs
        X = ns.velocity_mesh.node_coordinates()
        u0 = np.concatenate([(1 - X[:, 1] ** 2) * (1 + 0.1 * inputs.normal(0, "ux", N)),
                             0.1 * (1 - X[:, 1] ** 2) * inputs.normal(0, "uy", N),
                             0.1 * (1 - X[:, 1] ** 2) * inputs.normal(0, "uz", N)])
        ns.set_velocity(torch.tensor(u0, device="cuda"))
        f = (2 * nu, 0.0, 0.0)
        stats = [ns.step(f) for _ in range(max(args.warmup, 3))]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        stats = [ns.step(f) for _ in range(args.steps)]
        torch.cuda.synchronize()
        t = (time.perf_counter() - t0) / args.steps
        mean = lambda key: float(np.mean([st_[key] for st_ in stats]))
        out["dual_splitting_step"] = {
            "mesh": "%dx%dx%d tanh channel, k=%d" % (tuple(n_ns) + (w["k"],)), "velocity_dofs": 3 * N,
            "ms_per_step": 1e3 * t, "velocity_dof_steps_per_s": 3 * N / t, "steps_timed": args.steps,
            "pressure_iters": mean("pressure_iters"), "viscous_iters": mean("viscous_iters"),
            "projection_max_cell_iters": mean("projection_iters"), "nu": nu, "dt": dt, "order": 3,
            "rtol_pressure_viscous": 1e-6}
    elif args.workload == "perturbed":
        # the general-metric path: the 32^3 box with a smooth displacement,
        # k = 4, FP64 Laplace apply with the metric stored per quadrature point
        n_p = (args.cells,) * 3 if args.cells else (32, 32, 32)
        kp = args.k if args.k else 4
        m = Mesh(n_p, (0.0, -1.0, 0.0), (2 * math.pi, 1.0, math.pi), ("periodic", "dirichlet", "periodic"),
                 ("periodic", "dirichlet", "periodic"), mapping="perturbed", k=kp, amplitude=0.05,
                 seed=0x1234_5678_9ABC)
        m.set_f64_arithmetic(args.f64)
        N = m.n_dofs
        x = torch.tensor(inputs.uniform(0, "x", N), device="cuda")
        y = torch.empty_like(x)
        t, _ = _timed(lambda: [apply_laplace_f64(m, x, y) for _ in range(10)], reps=5)
        t /= 10
        p3 = (kp + 1) ** 3
        geo_bytes = 7 * 8 + 6 * 4 * 8 * (kp + 1) ** 2 / p3  # per DoF: cell metric + face data
        out["apply_general_f64"] = {"mesh": "%dx%dx%d perturbed box, k=%d" % (tuple(n_p) + (kp,)), "dofs": N,
                                    "ms": 1e3 * t, "dofs_per_s": N / t,
                                    "algorithmic_bytes_per_dof": 16 + geo_bytes,
                                    "achieved_gbs": N * (16 + geo_bytes) / t / 1e9}
    elif args.workload == "mg_scaling":
        # iteration counts of FP32-multigrid PCG (Sec. 5.1) and Jacobi PCG to
        # 1e-10 on refined channels: graded (tanh, gamma 1.8 / 0.9 / 0.3),
        # straight cells on the graded vertices, and the uniform box, k = 4,
        # seeded uniform rhs
        from paper_1607_01323_gb300 import Mesh as M_
        rows = []
        for mapping, gamma in (("channel", 1.8), ("channel_linear", 1.8), ("channel", 0.9), ("channel", 0.3),
                               ("affine", 1.8)):
            for n in (8, 16, 32):
                m = M_((n, n, n), w["lo"], w["hi"], w["bc_lo"], w["bc_hi"], mapping=mapping, gamma=gamma, k=4)
                b = torch.tensor(inputs.uniform(0, "b", m.n_dofs), device="cuda")
                _, rg = cg_solve(m, b, precond="gmg_f32", rtol=1e-10)
                _, rj = cg_solve(m, b, precond="jacobi", rtol=1e-10, maxit=20000)
                rows.append({"mapping": mapping, "gamma": gamma, "n": n, "gmg_iters": rg.iters,
                             "jacobi_iters": rj.iters})
        out["mg_scaling_k4"] = rows
    elif args.workload == "v3c":
        # the pressure-projection neighbours of the Poisson solve (variant V3c)
        # on the 32^3 k=4 channel: divergence rhs, pressure gradient, tau_D
        # and the div-div local projection; velocity = laminar profile + noise
        from paper_1607_01323_gb300 import (apply_divdiv_f64, apply_divergence_f64, apply_gradient_f64,
                                            project_divdiv_f64, tau_div_f64)
        m = Mesh(w["n"], w["lo"], w["hi"], w["bc_lo"], w["bc_hi"], mapping=w["mapping"], gamma=w["gamma"], k=w["k"])
        N = m.n_dofs
        X = m.node_coordinates()
        ux = (1 - X[:, 1] ** 2) + 0.1 * inputs.normal(0, "ux", N)
        u = torch.tensor(np.concatenate([ux, 0.1 * inputs.normal(0, "uy", N), 0.1 * inputs.normal(0, "uz", N)]),
                         device="cuda")
        pr = torch.tensor(inputs.uniform(0, "p", N), device="cuda")
        dt, gamma0 = 1e-3, 1.5
        yd = torch.empty(N, dtype=torch.float64, device="cuda")
        yg = torch.empty(3 * N, dtype=torch.float64, device="cuda")
        t_d, _ = _timed(lambda: [apply_divergence_f64(m, u, yd) for _ in range(20)], reps=3)
        t_g, _ = _timed(lambda: [apply_gradient_f64(m, pr, yg) for _ in range(20)], reps=3)
        tau = tau_div_f64(m, u, 1.0, dt)  # zeta_D = zeta* / CFL with zeta* = CFL = 1
        t_t, _ = _timed(lambda: [tau_div_f64(m, u, 1.0, dt, tau) for _ in range(20)], reps=3)
        rhs = apply_mass_f64(m, u) + (dt / gamma0) * apply_gradient_f64(m, pr)
        t_p, (xp, iters) = _timed(lambda: project_divdiv_f64(m, tau, rhs, rtol=1e-8, maxit=500), reps=3)
        res = apply_divdiv_f64(m, tau, xp) - rhs
        out["dofs_per_component"] = N
        out["divergence"] = {"ms": 1e3 * t_d / 20, "dofs_per_s": 3 * N / (t_d / 20)}
        out["gradient"] = {"ms": 1e3 * t_g / 20, "dofs_per_s": 3 * N / (t_g / 20)}
        out["tau_div"] = {"ms": 1e3 * t_t / 20, "mean": tau.mean().item(), "max": tau.max().item()}
        out["divdiv_projection"] = {"s": t_p, "max_cell_iters": iters, "rtol": 1e-8,
                                    "rel_residual": (torch.linalg.norm(res) / torch.linalg.norm(rhs)).item(),
                                    "dofs_per_s": 3 * N / t_p}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", default="solve", choices=["solve", "apply", "vcycle", "convective", "solve_only"],
                    help="apply: only operator applies; vcycle: only multigrid V-cycles; convective: only "
                         "convective-term applies; solve_only: only CG solves of the bench problem")
    ap.add_argument("--oracle-seconds", type=float, default=6.0,
                    help="seconds of sampled oracle applies per measurement of --workload oracle")
    ap.add_argument("--precond", default="jacobi", choices=["jacobi", "gmg_f32", "none", "invmass"],
                    help="preconditioner of --mode solve_only")
    ap.add_argument("--precision", default="f64", choices=["f64", "f32"])
    ap.add_argument("--cells", type=int, default=0)
    ap.add_argument("--k", type=int, default=0)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--f64", default="native", choices=["native", "double_float"],
                    help="arithmetic of the FP64 operator of the timed solves (native FP64, the default, or "
                         "double_float: FP32 pairs on the FP32 pipes)")
    ap.add_argument("--workload", default="c2",
                    choices=["c1", "c2", "c3", "c4", "c5", "v3c", "ns", "perturbed", "mg_scaling", "oracle"],
                    help="c2 (default) is the bench step; c1, c3-c5, v3c, ns print timings of other workloads")
    args = ap.parse_args()
    if args.mode == "apply":
        run_apply_only(args)
    elif args.mode == "vcycle":
        run_vcycle_only(args)
    elif args.mode == "convective":
        run_convective_only(args)
    elif args.mode == "solve_only":
        run_solve_only(args)
    elif args.workload == "oracle":
        run_oracle_timings(args)
    elif args.workload != "c2":
        run_config(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
