"""Benchmark: element-updates/s of one full elastic ADER-DG step at order 6 on 1,000,000
tetrahedra (CK derivatives + time integral + volume + local flux + neighbour flux), FP64,
synthetic SeisSol-reproducer-like inputs (random material, random affine elements, random
face matching with random orientations, DOFs ~ N(0,1)).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` is device-resident throughput (inputs in HBM);
`e2e` runs the same step through the C ABI with pinned host buffers (yt_step_host: H2D of
Q, step, D2H of Q, the copies pipelined with the kernels in element chunks).
`--impl reference` times the FP64 oracle on the host cores on a bounded sample.
Under torchrun (N > 1) every rank solves its own independent problem of the same size
(weak scaling, no data-path collective); the timed region is bracketed by barriers and the
maximum time over ranks is reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workload as wl  # noqa: E402

ORDER = 6
N_ELEMENTS = 1_000_000
METRIC = "element-updates/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 FMA peak derived from the unit counts and clocks of the part: 152 SMs x 2 FP64 FMA
# per clock per SM x 2 flop x 2070 MHz = 1.2586 TFLOP/s (nominal FP64: 1.25 TFLOP/s).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# FP32 FMA peak from the same unit counts: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# ncu DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of k_local per element,
# from one capture of a 40,000-tet case per order, keyed by the sha256 prefix of the
# kernel source it was captured on
NCU_TRAFFIC_PER_ELEMENT = {"3ad3ac46788ac2a3": {6: (304.467968e6 + 752.930816e6) / 40000},
                           "bb946a385f456ce8": {7: (411.153408e6 + 1193.212160e6) / 40000}}


def kernel_source_digest(order=6, precision="f64"):
    """Digest of what the timed kernels of one order and contraction type are built from:
    the kernel header and the generated rows and units of that degree, with comments and
    blank space removed (a comment edit does not change the kernels)."""
    h = hashlib.sha256()
    n = order - 1
    pkg = os.path.join(ROOT, "paper_1903_11521_gb300")
    files = [os.path.join(pkg, "csrc", "ader_kernels.cuh"), os.path.join(pkg, "csrc", "fp_convert.cuh"),
             os.path.join(pkg, "_build", "gen", f"yt_rows_o{n}.cuh")]
    files += [os.path.join(pkg, "_build", "gen", f"ader_o{n}_{precision}_{v}.cu") for v in ("lf", "nf")]
    for f in files:
        text = open(f).read() if os.path.exists(f) else "missing"
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update("".join(text.split()).encode())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--elements", type=int, default=N_ELEMENTS)
    ap.add_argument("--order", type=int, default=ORDER)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="f64", choices=["f64", "f32", "bf16x3"],
                    help="contraction type of the main measurement (default FP64)")
    ap.add_argument("--form", default=None,
                    choices=["executor", "structured", "viscoelastic", "serving", "local_update"],
                    help="run only this form of the forms section and print it as one JSON line "
                         "(for profiling one form)")
    ap.add_argument("--form-steps", type=int, default=10,
                    help="steps of the 27-quantity form at full size (--form viscoelastic)")
    ap.add_argument("--form-n", type=int, default=55,
                    help="cubes per direction of the 27-quantity form's mesh (--form viscoelastic; "
                         "55: 998,250 tets; smaller for profiling)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the precision, batching and serving measurements")
    return ap.parse_args()


def workload_config(args, extra=None):
    o = args.order
    B, BT = o * (o + 1) * (o + 2) // 6, o * (o + 1) // 2
    # bytes a step touches per element: Q and I (binary64), face projections and local
    # flux products (contraction type)
    rb = 8 if args.precision == "f64" else 4
    working = args.elements * (2 * 8 * 9 * B + 2 * rb * 4 * 9 * BT)
    cfg = {"workload": f"elastic ADER-DG full step, order {o} (B={B} x 9 quantities), "
                       f"{args.elements} tets, random 4-regular face matching",
           "order": o, "elements": args.elements, "quantities": 9,
           "precision": args.precision, "seed": wl.SEED,
           "l2": f"per-step working set (Q, I, face projections, local flux products: "
                 f"{working / 1e9:.1f} GB) exceeds the 129 MB L2 (no flush needed)"}
    if extra:
        cfg.update(extra)
    return cfg


# ---------------------------------------------------------------------- clocks sampler
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
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
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------- oracle baseline
def _oracle_local(args):
    from oracle import scheme
    Q, star, loc, dt, N = args
    _, I = scheme.derivatives_and_time_integral(Q, star, dt, N)
    return scheme.local_update(Q, I, star, loc, N), I


def _oracle_neigh(args):
    from oracle import scheme
    Qp, I, fnb, nb, fj, fh, N = args
    return scheme.neighbour_update(Qp, I, fnb, nb, fj, fh, N)


class OracleStep:
    """The FP64 oracle step (oracle.scheme, unmodified) over a sample of the workload,
    spread over the host cores by a spawn-started process pool (chunks of elements)."""

    def __init__(self, n_sample: int, order: int, workers: int):
        from oracle import basis, scheme
        N = order - 1
        self.N = N
        self.E = n_sample
        el = wl.random_elements(n_sample)
        self.conn = wl.random_connectivity(n_sample)
        self.Q = wl.random_dofs(n_sample, basis.n_basis(N), elements=el)
        self.dt = wl.cfl_time_step(el, N)
        self.star, self.loc, self.fnb = scheme.setup_element_matrices(el.rho, el.lam, el.mu, el.jac)
        basis.float_matrices(N)
        self.workers = workers
        self.pool = mp.get_context("spawn").Pool(workers, initializer=_pool_init, initargs=(N,))
        self.chunks = np.array_split(np.arange(n_sample), workers)

    def step(self):
        c = self.chunks
        res = self.pool.map(_oracle_local, [(self.Q[i], self.star[i], self.loc[i], self.dt, self.N) for i in c])
        Qp = np.concatenate([r[0] for r in res])
        I = np.concatenate([r[1] for r in res])
        # each chunk receives the time integrals of its own neighbours only
        jobs = []
        for i in c:
            nb = self.conn.neighbours[i]
            local_ids = np.arange(nb.size, dtype=np.int64).reshape(nb.shape)
            jobs.append((Qp[i], I[nb.ravel()], self.fnb[i], local_ids,
                         self.conn.faces[i], self.conn.orient[i], self.N))
        res2 = self.pool.map(_oracle_neigh, jobs)
        return np.concatenate(res2)

    def close(self):
        self.pool.close()
        self.pool.join()


def _pool_init(N):
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import basis
    basis.float_matrices(N)


def oracle_rate(order, target_s=12.0, workers=None):
    """Oracle element-updates/s on a sample sized for ~target_s seconds of CPU work."""
    workers = workers or os.cpu_count() or 1
    n = 256 * workers
    probe = OracleStep(n, order, workers)
    probe.step()
    t0 = time.perf_counter()
    probe.step()
    t = time.perf_counter() - t0
    probe.close()
    n2 = int(min(200_000, max(n, n * target_s / max(t, 1e-3))))
    runner = OracleStep(n2, order, workers)
    t0 = time.perf_counter()
    runner.step()
    t = time.perf_counter() - t0
    runner.close()
    return n2 / t, n2, t, workers


# ------------------------------------------------------------------------ forms
def _timed(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(steps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def _increment_error(yt, order, precision, n=20000):
    """Max over quantities of the relative Frobenius error of Q_new - Q against the FP64
    path (itself equal to the oracle to 1e-12) after one step on n elements."""
    N = order - 1
    B = order * (order + 1) * (order + 2) // 6
    el = wl.random_elements(n, seed=77)
    conn = wl.random_connectivity(n, seed=78)
    Q = wl.random_dofs(n, B, seed=79, scale="impedance", elements=el)
    dt = wl.cfl_time_step(el, N)
    mat = np.stack([el.rho, el.lam, el.mu], 1)
    out = []
    for prec in (yt.YT_F64, precision):
        s = yt.Solver(order, dt, mat, el.jac, conn.neighbours, conn.faces, conn.orient, precision=prec)
        s.set_dofs_host(Q)
        s.step()
        out.append(s.get_host() - Q)
        s.close()
    num = np.sqrt(((out[1] - out[0]) ** 2).sum((0, 1)))
    return float((num / np.sqrt((out[0] ** 2).sum((0, 1)))).max())


PRECISION_NAMES = {"f64": "FP64", "f32": "FP32", "bf16x3": "split-BF16 tensor-core (hi+lo, 3 products, FP32 accumulation)"}


def precision_code(yt, name):
    return {"f64": yt.YT_F64, "f32": yt.YT_F32, "bf16x3": yt.YT_BF16X3_F32ACC}[name]


def form_precision(yt, order, E, steps, stream, precision="f32"):
    N = order - 1
    B = order * (order + 1) * (order + 2) // 6
    el = wl.random_elements(E, seed=wl.SEED + 500)
    conn = wl.random_connectivity(E, seed=wl.SEED + 502)
    Q = wl.random_dofs(E, B, seed=wl.SEED + 501)
    dt = wl.cfl_time_step(el, N)
    code = precision_code(yt, precision)
    s = yt.Solver(order, dt, np.stack([el.rho, el.lam, el.mu], 1), el.jac, conn.neighbours,
                  conn.faces, conn.orient, precision=code, stream=stream)
    s.set_dofs_host(Q, stream=stream)
    ms = _timed(lambda: s.step(stream=stream), steps, 2, stream)
    s.status(stream=stream)
    st = s.stats()
    s.close()
    out = {"workload": f"order {order}, {E} tets, {PRECISION_NAMES[precision]} contractions / "
                       f"FP64 setup, accumulation and DOFs",
           "value": E / (ms / 1e3), "unit": METRIC, "ms_per_step": ms}
    # the step against the HBM roofline: algorithmic bytes (each stream once, the library's
    # count) over the measured copy bandwidth
    step_bytes = (st["local_bytes"] + st["neighbour_bytes"]) * E
    gbs = step_bytes / (ms / 1e3) / 1e9
    out["hbm"] = {"bytes_per_element": st["local_bytes"] + st["neighbour_bytes"], "achieved_gbs": gbs,
                  "peak_gbs": measured_hbm_gbs(), "frac": gbs / measured_hbm_gbs(),
                  "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth), of measured"}
    out["error_vs_fp64_increment"] = _increment_error(yt, order, code)
    out["error_definition"] = ("max over quantities of ||dQ - dQ_f64||_F / ||dQ_f64||_F, "
                               "one step, 20000 tets, against the FP64 path")
    return out


def measured_hbm_gbs():
    """HBM copy bandwidth of the measured peaks file, else the fallback figure (6.8 TB/s)."""
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def mass_diagonal(yt, order):
    """Diagonal of the library's reference mass matrix (the basis is orthogonal; the
    library returns M as its B diagonal entries)."""
    B = order * (order + 1) * (order + 2) // 6
    m = yt.reference_matrix(order, "M")
    return m if m.size == B else np.diag(m.reshape(B, B))


def elastic_energy(q, el, Mk, chunk=65536):
    """Elastic energy 1/2 int (rho |v|^2 + sigma : S sigma) of DOFs q (E, B, >= 9): the mass
    matrix of the basis is diagonal, so per element it is
    1/2 |J| sum_k M_kk (rho |v_k|^2 + sigma_k : S sigma_k), S the isotropic compliance:
    sigma : S sigma = (sigma : sigma - lambda / (3 lambda + 2 mu) tr(sigma)^2) / (2 mu)."""
    det = np.abs(np.linalg.det(el.jac))
    tot = 0.0
    for i in range(0, q.shape[0], chunk):
        d = q[i:i + chunk]
        rho, lam, mu = el.rho[i:i + chunk, None], el.lam[i:i + chunk, None], el.mu[i:i + chunk, None]
        ss = (d[..., 0:3] ** 2).sum(-1) + 2.0 * (d[..., 3:6] ** 2).sum(-1)
        tr = d[..., 0:3].sum(-1)
        dens = rho * (d[..., 6:9] ** 2).sum(-1) + (ss - lam / (3 * lam + 2 * mu) * tr ** 2) / (2 * mu)
        tot += 0.5 * float((det[i:i + chunk, None] * Mk[None, :] * dens).sum())
    return tot


def form_structured(yt, stream, n=55, steps=100):
    """100 steps on a jittered periodic structured mesh of n^3 cubes x 6 tets (n = 55:
    998,250 tets; vertices moved by up to 0.1 h, homogeneous material at the middle of the
    recipe's ranges, impedance-scaled N(0,1) DOFs, dt at CFL 0.5): orders 7 and 6 in FP64,
    FP32 and split-bf16 tensor-core contractions, each form from the same DOFs;
    the error of each reduced-precision form after 100 steps against the FP64 path.  No
    warm-up steps (every form must take the same 100 steps; solver creation has already
    run the setup kernel)."""
    mesh = wl.jittered_periodic_mesh(n, jitter=0.1, seed=wl.SEED + 800, length=100.0 * n,
                                     rho=2500.0, lam=2.5e10, mu=2.5e10)
    el, conn = mesh.elements, mesh.conn
    E = el.rho.size
    mat = np.stack([el.rho, el.lam, el.mu], 1)
    out = {"workload": f"jittered periodic structured mesh, {n}^3 cubes x 6 = {E} tets, "
                       f"vertex jitter 0.1 h, homogeneous material, {steps} steps"}

    def run(order, prec, Q0, warmup):
        dt = wl.cfl_time_step(el, order - 1)
        s = yt.Solver(order, dt, mat, el.jac, conn.neighbours, conn.faces, conn.orient,
                      precision=prec, stream=stream)
        s.set_dofs_host(Q0, stream=stream)
        ms = _timed(lambda: s.step(stream=stream), steps, warmup, stream)
        s.status(stream=stream)
        q = s.get_host(stream=stream)
        s.close()
        return ms, q

    def sq_per_quantity(a, b=None, chunk=65536):
        # sum over elements and basis functions of (a - b)^2 per quantity, in element
        # chunks (bounded host temporaries at order 7: a is 6 GB)
        acc = np.zeros(a.shape[-1])
        for i in range(0, a.shape[0], chunk):
            d = a[i:i + chunk] if b is None else a[i:i + chunk] - b[i:i + chunk]
            acc += np.einsum('ebq,ebq->q', d, d)
        return acc

    def energy(q, order):
        return elastic_energy(q, el, mass_diagonal(yt, order))

    def compare(order, forms):
        B = order * (order + 1) * (order + 2) // 6
        Q0 = wl.random_dofs(E, B, seed=wl.SEED + 800 + order, scale="impedance", elements=el)
        ms64, q64 = run(order, yt.YT_F64, Q0, 0)
        change = np.sqrt(sq_per_quantity(q64, Q0).sum())
        norm = np.sqrt(sq_per_quantity(q64).sum())
        res = {"fp64": {"value": E / (ms64 / 1e3), "unit": METRIC, "ms_per_step": ms64,
                        "finite": bool(np.isfinite(norm)),
                        "energy_ratio": energy(q64, order) / energy(Q0, order),
                        "coefficient_norm_ratio": float(norm / np.sqrt(sq_per_quantity(Q0).sum()))}}
        for name, prec in forms:
            ms, q = run(order, prec, Q0, 0)
            per_q = np.sqrt(sq_per_quantity(q, q64))
            res[name] = {"value": E / (ms / 1e3), "unit": METRIC, "ms_per_step": ms,
                         "error_vs_fp64_rel_solution": float(per_q.max() / norm),
                         "error_vs_fp64_rel_change": float(per_q.max() / change),
                         "energy_ratio": energy(q, order) / energy(Q0, order)}
            del q
        return res

    out["order7"] = compare(7, (("fp32", yt.YT_F32), ("bf16x3", yt.YT_BF16X3_F32ACC)))
    out["order6"] = compare(6, (("fp32", yt.YT_F32), ("bf16x3", yt.YT_BF16X3_F32ACC)))
    out["error_definition"] = ("after 100 steps from the same DOFs: max over quantities of "
                               "||Q - Q_fp64||_F, divided by ||Q_fp64||_F (rel_solution) or by "
                               "||Q_fp64 - Q_0||_F (rel_change); energy_ratio = elastic energy "
                               "1/2 int(rho |v|^2 + sigma : S sigma) after the steps / before "
                               "(mass-weighted; below 1: the upwind flux dissipates)")
    return out


def form_viscoelastic(yt, stream, n=55, order=7, steps=10, n_long=20, steps_long=100):
    """The 27-quantity precision form: order 7, the jittered periodic structured mesh of
    n^3 x 6 tets (n = 55: 998,250), homogeneous elastic material, synthetic attenuation of
    three mechanisms per element (workload.attenuation), N(0,1) DOFs scaled by impedance
    (stresses) and impedance x omega (anelastic functions); FP64, FP32 and split-bf16
    tensor-core contractions, `steps` steps each from the same DOFs (no warm-up: all take
    the same steps), the reduced-precision results after them against the FP64 path (which equals the oracle to 1e-15 per step,
    tests/test_gpu_viscoelastic.py).  The error after `steps_long` steps is measured the same
    way on the n_long^3 x 6 mesh of the same family (100 FP64 steps at full size take
    two minutes)."""
    out = _viscoelastic_run(yt, stream, n, order, steps)
    if steps_long:
        long = _viscoelastic_run(yt, stream, n_long, order, steps_long)
        keys = ("error_vs_fp64_rel_solution", "error_vs_fp64_rel_change",
                "error_vs_fp64_rel_solution_elastic", "error_vs_fp64_rel_solution_anelastic")
        out["error_after_100_steps"] = {"workload": long["workload"], "fp64_finite": long["fp64"]["finite"]}
        for key in ("fp32", "bf16x3"):
            out["error_after_100_steps"][key] = {k: long[key][k] for k in keys}
    return out


def _viscoelastic_run(yt, stream, n, order, steps):
    mesh = wl.jittered_periodic_mesh(n, jitter=0.1, seed=wl.SEED + 800, length=100.0 * n,
                                     rho=2500.0, lam=2.5e10, mu=2.5e10)
    el, conn = mesh.elements, mesh.conn
    E = el.rho.size
    N = order - 1
    B = order * (order + 1) * (order + 2) // 6
    dt = wl.cfl_time_step(el, N)
    att = wl.attenuation(el, dt, seed=wl.SEED + 900)
    Q0 = wl.random_dofs_viscoelastic(E, B, el, att, seed=wl.SEED + 901)
    mat = np.stack([el.rho, el.lam, el.mu], 1)

    # full steps (phase 0, then phase 1), both phases timed with CUDA events
    def run_steps(prec):
        import torch
        s = yt.Solver(order, dt, mat, el.jac, conn.neighbours, conn.faces, conn.orient,
                      precision=prec, stream=stream, attenuation=att)
        s.set_dofs_host(Q0, stream=stream)
        st = s.stats()
        evs = [[torch_event() for _ in range(3)] for _ in range(steps)]
        torch.cuda.synchronize()
        for k in range(steps):
            evs[k][0].record(stream)
            s.step_phase(0, stream=stream)
            evs[k][1].record(stream)
            s.step_phase(1, stream=stream)
            evs[k][2].record(stream)
        torch.cuda.synchronize()
        total = evs[0][0].elapsed_time(evs[-1][2]) / steps
        loc = sum(e[0].elapsed_time(e[1]) for e in evs) / steps
        nei = sum(e[1].elapsed_time(e[2]) for e in evs) / steps
        q = s.get_host(stream=stream)
        s.close()
        return q, st, total, loc, nei

    def sq(a, b=None, chunk=32768):
        acc = np.zeros(a.shape[-1])
        for i in range(0, a.shape[0], chunk):
            d = a[i:i + chunk] if b is None else a[i:i + chunk] - b[i:i + chunk]
            acc += np.einsum('ebq,ebq->q', d, d)
        return acc

    out = {"workload": f"viscoelastic-shaped (3 mechanisms, 27 quantities), order {order} "
                       f"(B={B}), jittered periodic structured mesh {n}^3 x 6 = {E} tets, "
                       f"{steps} steps", "elements": E, "quantities": 27, "steps": steps}
    q64, st64, t64, l64, n64 = run_steps(yt.YT_F64)
    norm = np.sqrt(sq(q64))
    change = np.sqrt(sq(q64, Q0))
    out["fp64"] = {"value": E / (t64 / 1e3), "unit": METRIC, "ms_per_step": t64,
                   "kernel_ms": {"k_local": l64, "k_neigh+k_theta": n64},
                   "tflops": (st64["local_flops"] + st64["neighbour_flops"]) * E / (t64 / 1e3) / 1e12,
                   "frac_fp64_peak": (st64["local_flops"] + st64["neighbour_flops"]) * E / (t64 / 1e3) / 1e12
                   / FP64_PEAK_TFLOPS,
                   "finite": bool(np.isfinite(norm).all())}
    # the reduced-precision forms one after the other, each result compared and dropped
    # before the next runs (an order-7 27-quantity state of 1M tets is 18 GB on the host)
    for key, prec in (("fp32", yt.YT_F32), ("bf16x3", yt.YT_BF16X3_F32ACC)):
        qr, str_, tr, lr, nr = run_steps(prec)
        per_q = np.sqrt(sq(qr, q64))
        del qr
        out[key] = {"value": E / (tr / 1e3), "unit": METRIC, "ms_per_step": tr,
                    "kernel_ms": {"k_local": lr, "k_neigh+k_theta": nr},
                    "tflops": (str_["local_flops"] + str_["neighbour_flops"]) * E / (tr / 1e3) / 1e12,
                    "error_vs_fp64_rel_solution": float((per_q / norm).max()),
                    "error_vs_fp64_rel_change": float((per_q / change).max()),
                    "error_vs_fp64_rel_solution_elastic": float((per_q[:9] / norm[:9]).max()),
                    "error_vs_fp64_rel_solution_anelastic": float((per_q[9:] / norm[9:]).max())}
    out["bf16x3"]["contractions"] = ("elastic rows' global-matrix products on the tensor cores (split "
                                     "bf16, FP32 accumulation); anelastic rows FP32 CUDA cores")
    out["flops_per_element"] = {"local": st64["local_flops"], "neighbour_and_theta": st64["neighbour_flops"]}
    out["error_definition"] = (f"after {steps} steps from the same DOFs: max over the 27 quantities "
                               "of ||Q - Q_fp64||_F / ||Q_fp64||_F (rel_solution, the same restricted to "
                               "the 9 elastic and the 18 anelastic quantities) or / ||Q_fp64 - Q_0||_F "
                               "(rel_change)")
    return out


def torch_event():
    import torch
    return torch.cuda.Event(enable_timing=True)


def form_executor(yt, stream, order=6, E=200_000, S=8, reps=5):
    """The generic planner / batched executor (yt_plan_create + yt_execute_batched) on two
    of the step's contractions written as expressions, FP64, random per-element data:
    the volume kernel, and the neighbour-flux chain with S fused simulations (index s of
    the DOFs and time integral).  Global matrices from the library's reference matrices;
    star and flux-solver matrices dense per element."""
    import torch
    def matrices(o):
        B, BT = o * (o + 1) * (o + 2) // 6, o * (o + 1) // 2
        return (B, BT,
                yt.reference_matrix(o, "Khat").reshape(3, B, B).transpose(0, 2, 1),
                yt.reference_matrix(o, "R").reshape(4, BT, B).transpose(0, 2, 1),
                yt.reference_matrix(o, "Rhat").reshape(4, BT, B).transpose(0, 2, 1),
                yt.reference_matrix(o, "f").reshape(3, BT, BT).transpose(0, 2, 1))

    B, BT, Kh, R, Rh, f = matrices(order)
    gen = torch.Generator(device="cuda").manual_seed(wl.SEED + 900)

    def run(expr, consts, per_elem, n):
        tensors = [(name, shape, None, None) for name, shape in per_elem]
        tensors += [(name, val.shape, val != 0, val) for name, val in consts]
        plan = yt.Plan(expr, tensors, precision=yt.YT_F64)
        dev = {name: torch.randn((n, int(np.prod(shape))), dtype=torch.float64, device="cuda",
                                 generator=gen) for name, shape in per_elem}
        plan.execute(dev, n, stream=stream)           # warm-up (scratch sized here)
        ms = _timed(lambda: plan.execute(dev, n, stream=stream), reps, 1, stream)
        st = plan.stats()
        plan.close()
        del dev
        torch.cuda.empty_cache()
        tflops = st["nz_flops"] * n / (ms / 1e3) / 1e12
        return {"ms": ms, "elements_per_s": n / (ms / 1e3), "nz_flops_per_element": st["nz_flops"],
                "achieved_tflops": tflops, "frac_fp64_peak": tflops / FP64_PEAK_TFLOPS,
                "order_chosen": st["order"]}

    out = {"workload": f"generic executor, order {order}, FP64, random per-element data"}
    vol = run("V[kp] += K0[kl]*I[lq]*A0[pq] + K1[kl]*I[lq]*A1[pq] + K2[kl]*I[lq]*A2[pq]",
              [(f"K{x}", Kh[x]) for x in range(3)],
              [("I", (B, 9)), ("A0", (9, 9)), ("A1", (9, 9)), ("A2", (9, 9)), ("V", (B, 9))], E)
    vol["expression"] = "volume: V += sum_x Khat^x I A^xT"
    out["volume"] = vol
    nf = E // S
    # the planner picks the chain order from the sizes and the actual sparsity patterns of
    # these face matrices (reported as order_chosen)
    for o in (order, 4):
        Bo, BTo, _, Ro, Rho, fo = matrices(o)
        fused = run("G[kps] += Rh[km] * f[mn] * R[ln] * J[lqs] * An[pq]",
                    [("Rh", Rho[1]), ("f", fo[2]), ("R", Ro[3])],
                    [("J", (Bo, 9, S)), ("An", (9, 9)), ("G", (Bo, 9, S))], nf)
        fused["expression"] = (f"order {o}, neighbour flux of one face, {S} fused simulations: "
                               f"G += Rhat f R^T J A^T")
        fused["element_simulations_per_s"] = fused["elements_per_s"] * S
        out[f"neighbour_fused_simulations_o{o}"] = fused
    return out


def form_local_update(yt, order, E, steps, stream):
    """Local update alone (derivatives, time integral, volume, local flux; no neighbour
    flux) of a small mesh: order 4, 1,000 tets, FP64, N(0,1) DOFs."""
    N = order - 1
    B = order * (order + 1) * (order + 2) // 6
    el = wl.random_elements(E, seed=wl.SEED + 700)
    Q = wl.random_dofs(E, B, seed=wl.SEED + 701)
    dt = wl.cfl_time_step(el, N)
    s = yt.Solver(order, dt, np.stack([el.rho, el.lam, el.mu], 1), el.jac, stream=stream)
    s.set_dofs_host(Q, stream=stream)
    ms = _timed(lambda: s.step_local(stream=stream), steps, 10, stream)
    s.close()
    tiles = (E + 31) // 32
    return {"workload": f"local update (CK, time integral, volume, local flux), order {order}, "
                        f"{E} tets, FP64; meshes of at most one tile per SM run on CTAs of 8 tets "
                        f"({4 * tiles} CTAs here, the small-mesh kernel)",
            "value": E / (ms / 1e3), "unit": METRIC, "ms_per_step": ms}


def form_batching(yt, E, precision, lo, hi, steps, stream):
    rng = np.random.default_rng(wl.SEED + 600)
    orders = rng.integers(lo, hi + 1, E).astype(np.int8)
    el = wl.random_elements(E, seed=wl.SEED + 601)
    conn = wl.random_connectivity(E, seed=wl.SEED + 602)
    dt = wl.cfl_time_step(el, int(orders.max()) - 1)
    b = yt.Batch(orders, dt, np.stack([el.rho, el.lam, el.mu], 1), el.jac, conn.neighbours,
                 conn.faces, conn.orient, precision=precision, stream=stream)
    flat = rng.standard_normal(int(b.offsets[-1]))
    b._host_in = flat
    b.set_dofs_ptr(flat.ctypes.data, yt.YT_MEM_HOST, stream=stream)
    # every form timed on the same data (each from the same starting DOFs), then the
    # tuner's choice
    forms = {}
    for name, form, order, chunk in (("per_degree_kernels_sequence", 0, 0, 1),
                                     ("per_degree_kernels_branches", 1, 0, 1),
                                     ("persistent_by_degree_chunk1", 2, 0, 1)):
        b.set_form(form, order, chunk)
        b.set_dofs_ptr(flat.ctypes.data, yt.YT_MEM_HOST, stream=stream)
        forms[name] = _timed(lambda: b.step(stream=stream), steps, 2, stream)
    b.status(stream=stream)
    b.set_dofs_ptr(flat.ctypes.data, yt.YT_MEM_HOST, stream=stream)
    chosen = b.tune(3, stream=stream)
    ms = _timed(lambda: b.step(stream=stream), steps, 2, stream)
    b.status(stream=stream)
    st = b.stats()
    cfg = b.config()
    b.close()
    return {"workload": f"p-adaptive mesh, {E} tets, per-element order U{{{lo}..{hi}}}, "
                        f"{'FP32' if precision == yt.YT_F32 else 'FP64'}",
            "value": E / (ms / 1e3), "unit": METRIC, "ms_per_step": ms,
            "chosen_form": ["per-degree kernels in sequence", "per-degree kernels on parallel branches",
                            "persistent kernel"][chosen],
            "tuner": cfg, "ms_per_step_by_form": forms,
            "groups": st["groups"], "achieved_tflops": st["flops"] / (ms / 1e3) / 1e12}


def form_serving(yt, n_requests=256, rate=20.0, steps=100, budget=64 << 30):
    import threading as th
    rng = np.random.default_rng(wl.SEED + 700)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_requests))
    target = np.exp(rng.uniform(np.log(1e3), np.log(2e5), n_requests))
    orders = rng.integers(3, 7, n_requests)
    # every solve runs 100 steps, so its mesh must be a real mesh: the jittered periodic
    # structured mesh of n^3 x 6 tets with n^3 x 6 nearest to the drawn size (one mesh per
    # n, 1,296 .. 196,608 tets), homogeneous material, impedance-scaled N(0,1) DOFs
    ns = np.clip(np.rint((target / 6.0) ** (1.0 / 3.0)).astype(int), 6, 32)
    sizes = 6 * ns ** 3
    meshes = {}
    for n in sorted(set(int(x) for x in ns)):
        meshes[n] = wl.jittered_periodic_mesh(n, jitter=0.1, seed=wl.SEED + 750 + n, length=100.0 * n,
                                             rho=2500.0, lam=2.5e10, mu=2.5e10)
    reqs = []
    for i in range(n_requests):
        n, o = int(ns[i]), int(orders[i])
        el, conn = meshes[n].elements, meshes[n].conn
        E = el.rho.size
        Q = wl.random_dofs(E, o * (o + 1) * (o + 2) // 6, seed=wl.SEED + 10002 + 3 * i, scale="impedance",
                           elements=el)
        reqs.append((o, wl.cfl_time_step(el, o - 1), np.stack([el.rho, el.lam, el.mu], 1), el.jac,
                     conn.neighbours, conn.faces, conn.orient, Q))
    srv = yt.Server(budget, precision=yt.YT_F32)
    ids = [None] * n_requests
    t0 = time.perf_counter()

    def submitter():
        for i, r in enumerate(reqs):
            delay = arrivals[i] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            ids[i] = srv.submit(*r, steps)

    thread = th.Thread(target=submitter)
    thread.start()
    thread.join()
    subset = set(range(0, n_requests, 8))          # results kept for the FP64 comparison
    lat, queue, served = [], [], {}
    for i, rid in enumerate(ids):
        q_out, l, q = srv.wait(rid)
        lat.append(l)
        queue.append(q)
        if i in subset:
            served[i] = q_out
    t_end = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    lat = np.array(lat) * 1e3
    out = {"workload": f"{n_requests} independent elastic solves, Poisson arrivals {rate}/s, "
                       f"sizes log-U[1e3, 2e5] tets (jittered periodic meshes of n^3 x 6 tets, n = 6..32), "
                       f"orders U{{3..6}}, {steps} steps each, FP32 contractions / FP64 accumulation, "
                       f"HBM budget {budget >> 30} GiB",
           "solves_per_s": n_requests / t_end, "p50_latency_ms": float(np.percentile(lat, 50)),
           "p99_latency_ms": float(np.percentile(lat, 99)),
           "p50_queue_ms": float(np.percentile(np.array(queue) * 1e3, 50)),
           "element_updates_per_s": st["element_updates"] / t_end,
           "makespan_s": t_end, "max_active": st["max_active"], "peak_bytes": st["peak_bytes"],
           "completed": st["completed"], "failed": st["failed"]}
    # the plain path on the same stream: every solve alone on a plain solver of the same
    # precision (create, upload, the steps, download), one after another in arrival
    # order; service times measured, first-in-first-out queueing computed from them
    import torch
    service = []
    for r in reqs:
        torch.cuda.synchronize()
        t = time.perf_counter()
        s = yt.Solver(*r[:7], precision=yt.YT_F32)
        s.set_dofs_host(r[7])
        for _ in range(steps):
            s.step()
        s.get_host()
        s.close()
        service.append(time.perf_counter() - t)
    finish, plain_lat = 0.0, []
    for a, sv in zip(arrivals, service):
        finish = max(finish, a) + sv
        plain_lat.append(finish - a)
    plain_lat = np.array(plain_lat) * 1e3
    out["plain_one_at_a_time"] = {
        "solves_per_s": n_requests / finish, "p50_latency_ms": float(np.percentile(plain_lat, 50)),
        "p99_latency_ms": float(np.percentile(plain_lat, 99)),
        "element_updates_per_s": st["element_updates"] / finish, "makespan_s": finish,
        "busy_s": float(np.sum(service))}
    # the plain FP64 path: every 8th request measured alone in FP64 (its final DOFs kept);
    # the error of the served FP32 result of the same request against it; the FP64
    # service time of every request from a per-order fit t = a + b E of the measured ones,
    # and first-in-first-out queueing on the same arrivals from those times
    svc64, errs = {}, []
    for i in sorted(subset):
        r = reqs[i]
        torch.cuda.synchronize()
        t = time.perf_counter()
        s = yt.Solver(*r[:7], precision=yt.YT_F64)
        s.set_dofs_host(r[7])
        for _ in range(steps):
            s.step()
        q64 = s.get_host()
        s.close()
        svc64[i] = time.perf_counter() - t
        num = np.sqrt(((served[i] - q64) ** 2).sum((0, 1)))
        errs.append(float((num / np.sqrt((q64 ** 2).sum((0, 1)))).max()))
        del q64
    fit = {}
    for o in sorted(set(int(x) for x in orders)):
        idx = [i for i in svc64 if int(orders[i]) == o]
        A = np.stack([np.ones(len(idx)), sizes[idx].astype(float)], 1)
        fit[o] = np.linalg.lstsq(A, np.array([svc64[i] for i in idx]), rcond=None)[0]
    pred = [svc64.get(i, float(fit[int(orders[i])][0] + fit[int(orders[i])][1] * sizes[i]))
            for i in range(n_requests)]
    finish64, lat64 = 0.0, []
    for a, sv in zip(arrivals, pred):
        finish64 = max(finish64, a) + sv
        lat64.append(finish64 - a)
    lat64 = np.array(lat64) * 1e3
    out["plain_fp64_one_at_a_time"] = {
        "solves_per_s": n_requests / finish64, "p50_latency_ms": float(np.percentile(lat64, 50)),
        "p99_latency_ms": float(np.percentile(lat64, 99)), "makespan_s": finish64,
        "busy_s": float(np.sum(pred)), "measured_solves": len(svc64),
        "method": f"{len(svc64)} of the {n_requests} requests (every 8th) run alone in FP64 and timed; "
                  "the others' service times from a per-order fit t = a + b E of those; FIFO queueing "
                  "on the same arrivals"}
    out["served_fp32_error_vs_fp64"] = {
        "max": max(errs), "median": float(np.median(errs)), "requests": len(errs),
        "definition": f"after {steps} steps: max over quantities of ||Q_served - Q_fp64||_F / ||Q_fp64||_F, "
                      "the same request run alone in FP64"}
    return out


# ------------------------------------------------------------------------ GPU bench
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    import paper_1903_11521_gb300 as yt

    if args.form:
        stream = torch.cuda.current_stream()
        run = {"executor": lambda: form_executor(yt, stream),
               "structured": lambda: form_structured(yt, stream),
               "viscoelastic": lambda: form_viscoelastic(yt, stream, n=args.form_n, steps=args.form_steps,
                                                         steps_long=0 if args.form_n != 55 else 100),
               "serving": lambda: form_serving(yt),
               "local_update": lambda: form_local_update(yt, 4, 1000, 200, stream)}[args.form]
        print(json.dumps({"form": args.form, "result": run()}), flush=True)
        return

    N = args.order - 1
    B = args.order * (args.order + 1) * (args.order + 2) // 6
    E = args.elements
    stream = torch.cuda.current_stream()
    prec = precision_code(yt, args.precision)
    part = None
    if ws > 1:
        # one mesh of ws x E elements (the same recipe) partitioned in blocks: E per rank,
        # one halo exchange of face projections per step over NCCL
        from paper_1903_11521_gb300 import partition
        el = wl.random_elements(ws * E, seed=wl.SEED)
        conn = wl.random_connectivity(ws * E, seed=wl.SEED + 2)
        dt = wl.cfl_time_step(el, N)
        import torch.distributed as dist
        part = partition.PartitionedSolver(args.order, dt, el, conn, partition.block_partition(ws * E, ws),
                                           rank, dist, precision=prec, stream=stream, staging="device")
        Q = wl.random_dofs(part.ids.size, B, seed=wl.SEED + 1 + 1000 * rank)
        part.set_dofs_local(Q)
        solver = part.solver
        E = part.ids.size
    else:
        el = wl.random_elements(E, seed=wl.SEED)
        conn = wl.random_connectivity(E, seed=wl.SEED + 2)
        Q = wl.random_dofs(E, B, seed=wl.SEED + 1)
        dt = wl.cfl_time_step(el, N)
        solver = yt.Solver(args.order, dt, np.stack([el.rho, el.lam, el.mu], 1), el.jac,
                           conn.neighbours, conn.faces, conn.orient, precision=prec, stream=stream)
        solver.set_dofs_host(Q, stream=stream)
    torch.cuda.synchronize()
    stats = solver.stats()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def full_step():
        if part is not None:
            part.step()
        else:
            solver.step(stream=stream)

    def rest_of_step():
        # phase 1: with a partition, the halo gather, the neighbour kernel of the interior
        # tiles, the exchange and the neighbour kernel of the boundary tiles
        if part is None:
            solver.step_phase(1, stream=stream)
            return
        if sum(part.send_counts):
            solver.halo_pack(part.send_buf.data_ptr(), stream=stream)
        solver.step_phase_tiles(1, 0, part.n_interior_tiles, stream=stream)
        part._exchange()
        if part.n_halo:
            solver.halo_unpack(part.recv_buf.data_ptr(), stream=stream)
        solver.step_phase_tiles(1, part.n_interior_tiles, part.n_tiles - part.n_interior_tiles, stream=stream)

    # kernels of one timed step: k_local and k_neigh; with a partition the halo gather,
    # the halo scatter, and k_neigh split into the interior and the boundary tiles
    launches_per_step = 2
    if part is not None:
        launches_per_step = (1 + int(sum(part.send_counts) > 0) + int(part.n_interior_tiles > 0)
                             + int(part.n_halo > 0) + int(part.n_tiles > part.n_interior_tiles))
    for _ in range(args.warmup):
        full_step()
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.5)
    barrier()
    for k in range(K):
        ev[k][0].record(stream)
        solver.step_phase(0, stream=stream)
        ev[k][1].record(stream)
        rest_of_step()
        ev[k][2].record(stream)
    barrier()
    clk = clocks.stop()
    total_ms = ev[0][0].elapsed_time(ev[K - 1][2])
    local_ms = sum(e[0].elapsed_time(e[1]) for e in ev) / K
    neigh_ms = sum(e[1].elapsed_time(e[2]) for e in ev) / K
    step_ms = sorted(e[0].elapsed_time(e[2]) for e in ev)
    t_max = total_ms
    if ws > 1:
        import torch.distributed as dist
        tt = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
    value = ws * E * K / (t_max / 1e3)

    # end to end through the C ABI with host buffers (pinned), H2D + step + D2H per step
    e2e = None
    if not args.no_e2e and part is None:
        canon = torch.empty((E, 9, B), dtype=torch.float64, pin_memory=True)
        canon.numpy()[:] = Q.transpose(0, 2, 1)
        out = torch.empty_like(canon, pin_memory=True)
        for _ in range(2):
            solver.step_host_ptr(canon.data_ptr(), out.data_ptr(), stream=stream)
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(K):
            solver.step_host_ptr(canon.data_ptr(), out.data_ptr(), stream=stream)
        b.record(stream)
        barrier()
        e_ms = a.elapsed_time(b)
        if ws > 1:
            import torch.distributed as dist
            tt = torch.tensor([e_ms], device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            e_ms = float(tt.item())
        nbytes = E * 9 * B * 8
        # the copies alone (one each way, pinned host <-> device, on the same stream)
        dev = torch.empty(canon.shape, dtype=canon.dtype, device="cuda")
        c0, c1, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        torch.cuda.synchronize()
        c0.record(stream)
        dev.copy_(canon, non_blocking=True)
        c1.record(stream)
        out.copy_(dev, non_blocking=True)
        c2.record(stream)
        torch.cuda.synchronize()
        h2d_ms, d2h_ms = c0.elapsed_time(c1), c1.elapsed_time(c2)
        del dev
        seq_ms = h2d_ms + total_ms / K + d2h_ms
        e2e = {"value": ws * E * K / (e_ms / 1e3), "unit": METRIC,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "ms_per_step": e_ms / K,
               "h2d_gbs": nbytes / (h2d_ms / 1e3) / 1e9, "d2h_gbs": nbytes / (d2h_ms / 1e3) / 1e9,
               "copy_ms_alone": [h2d_ms, d2h_ms],
               "sequential_ms": seq_ms,
               "overlap_fraction": max(0.0, min(1.0, (seq_ms - e_ms / K) / (h2d_ms + d2h_ms))),
               "overlap_definition": "(H2D + device step + D2H, each alone) - e2e step, over the "
                                     "copy time: the share of the copies hidden under the kernels"}
    if not args.no_e2e and part is not None:
        # partitioned: every step uploads this rank's DOFs from pinned host memory, runs
        # the partitioned step (with its exchange) and downloads the result
        canon = torch.empty((E, 9, B), dtype=torch.float64, pin_memory=True)
        canon.numpy()[:] = Q.transpose(0, 2, 1)
        out = torch.empty_like(canon, pin_memory=True)

        def host_step():
            solver.set_dofs_ptr(canon.data_ptr(), yt.YT_MEM_HOST, stream=stream)
            part.step()
            solver.get_ptr(yt.YT_FIELD_DOFS, out.data_ptr(), yt.YT_MEM_HOST, stream=stream)
        host_step()
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(K):
            host_step()
        b.record(stream)
        barrier()
        e_ms = a.elapsed_time(b)
        import torch.distributed as dist
        tt = torch.tensor([e_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e_ms = float(tt.item())
        nbytes = E * 9 * B * 8
        e2e = {"value": ws * E * K / (e_ms / 1e3), "unit": METRIC, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "ms_per_step": e_ms / K,
               "definition": "per rank: H2D of its DOFs, the partitioned step, D2H of its DOFs"}
    solver.close()

    if rank != 0:
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
            dist.destroy_process_group()
        return

    flops_local = stats["local_flops"] * E
    achieved = flops_local / (local_ms / 1e3) / 1e12
    peak = FP32_PEAK_TFLOPS if args.precision != "f64" else FP64_PEAK_TFLOPS
    peak_source = ("FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2070 MHz (derived)" if args.precision != "f64"
                   else "FP64 FMA: 152 SMs x 2 FMA/clk x 2 flop x 2070 MHz (derived)")
    roofline = {"bound": "alu", "kernel": "k_local (derivatives + time integral + volume + face projections + local flux products)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "peak_source": peak_source,
                "traffic": None,
                "k_neigh_frac": stats["neighbour_flops"] * E / (neigh_ms / 1e3) / 1e12 / peak,
                "step_frac": (stats["local_flops"] + stats["neighbour_flops"]) * E / (total_ms / K / 1e3) / 1e12 / peak,
                "flops_per_element": {"local": stats["local_flops"], "neighbour": stats["neighbour_flops"]}}
    # DRAM bytes per element of k_local from one ncu capture of a 40,000-tet case, valid
    # only for the kernel source it was taken on (scaled to E: traffic grows with E)
    digest = kernel_source_digest(args.order, args.precision)
    if args.precision == "f64" and args.order in NCU_TRAFFIC_PER_ELEMENT.get(digest, {}):
        roofline["traffic"] = NCU_TRAFFIC_PER_ELEMENT[digest][args.order] * E
        roofline["traffic_unit"] = "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum, scaled)"

    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        rate, n_s, t_s, cores = oracle_rate(args.order)
        cpu = {"value": rate, "unit": METRIC, "cores": cores, "kind": "oracle",
               "sample": f"{n_s} elements of the same workload recipe, one full step "
                         f"({t_s:.1f} s), dense unfactorised FP64 oracle"}
    forms = None
    if not args.no_forms and ws == 1:
        forms = {"local_update_o4_1000": form_local_update(yt, 4, 1000, 200, stream),
                 "precision_o6": form_precision(yt, 6, E, 5, stream),
                 "precision_o6_bf16x3": form_precision(yt, 6, E, 5, stream, "bf16x3"),
                 "precision_o7": form_precision(yt, 7, E, 5, stream),
                 "precision_o7_bf16x3": form_precision(yt, 7, E, 5, stream, "bf16x3"),
                 "structured_mesh_100_steps": form_structured(yt, stream),
                 "viscoelastic_o7": form_viscoelastic(yt, stream),
                 "executor": form_executor(yt, stream),
                 "batching_fp32": form_batching(yt, 2 * E, yt.YT_F32, 3, 7, 5, stream),
                 "batching_fp64": form_batching(yt, 2 * E, yt.YT_F64, 3, 7, 3, stream),
                 "serving": form_serving(yt)}
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": K,
            "warmup": args.warmup, "ms_per_step": t_max / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": workload_config(args, {"parallelism": (f"element partition over {ws} GPUs ({E} tets each, "
                                                             "one NCCL halo exchange of face projections per step)")
                                             if ws > 1 else "one GPU"}),
            "clocks": clk, "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu, "forms": forms,
            "gpu_launches": launches_per_step * K,
            "kernel_ms": {"k_local": local_ms, "k_neigh": neigh_ms},
            "step_ms_min_median": [step_ms[0], step_ms[len(step_ms) // 2]],
            "context": {"paper_skx_dp_o6_element_updates_per_s": 1244e6 / (56 * 9),
                        "paper_hardware": "2x Xeon Platinum 8174 (SKX), App. A"}}
    print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    workers = os.cpu_count() or 1
    # size one step of the oracle for ~8 s on the host cores
    rate, _, _, _ = oracle_rate(args.order, target_s=3.0, workers=workers)
    n = int(max(256 * workers, min(200_000, rate * 8.0)))
    runner = OracleStep(n, args.order, workers)
    for _ in range(args.warmup):
        runner.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        runner.step()
    t = time.perf_counter() - t0
    runner.close()
    value = n * args.steps / t
    sample = (f"{n} elements of the same workload recipe per step (the full problem has "
              f"{args.elements}); dense unfactorised FP64 oracle, spawn pool of {workers} processes")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, {"parallelism": (f"element partition over {ws} GPUs ({args.elements} "
                                                             "tets each, one NCCL halo exchange of face projections "
                                                             "per step)") if ws > 1 else "one GPU"}),
            "sample_elements": n,
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": workers, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
