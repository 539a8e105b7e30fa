#!/usr/bin/env python
"""Benchmark: Truncated Solver Method disconnected loops on one GB300.

One step = one complete TSM estimate (Sec. 2.1, Eq. 4) on the 32^3 x 64
workload: Z4 noise for N_HP + N_LP = 8 + 256 sources, low-precision (FP16)
CG solves of all of them truncated at |r|/|b| = 1e-2, mixed-precision CG of
the 8 high-precision sources to 1e-9 with FP64 reliable updates, local and
one-derivative loops with the one-end trick (Eq. 5) and its generalisation
(Eq. 6) for every solution, and the TSM combination.  The metric is seconds
per source (lower is better).

Prints one JSON line (rank 0).  Usage:
    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs its own disjoint set of sources (weak scaling).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CONFIGS = {
    # the paper's production volume and TSM layout (Secs. 2.1, 3), synthetic links
    "tsm32": dict(L=(32, 32, 32, 64), kappa=0.161, mu=0.003, n_hp=8, n_lp=256, batch=16,
                  lp_prec="f16", hp_inner="f32", tol_lp=1e-2, tol_hp=1e-9, gauge_seed=1237,
                  seed=20140126, schur=True, delta=3e-5, recon=0, overlap=False, hp_loops="ff", hp_ru="f64"),
    # the same layout on 24^3 x 48 (fields larger than L2): the size of the ncu captures
    "tsm24": dict(L=(24, 24, 24, 48), kappa=0.161, mu=0.003, n_hp=8, n_lp=24, batch=16,
                  lp_prec="f16", hp_inner="f32", tol_lp=1e-2, tol_hp=1e-9, gauge_seed=1237,
                  seed=20140126, schur=True, delta=3e-5, recon=0, overlap=False, hp_loops="ff", hp_ru="f64"),
    # small case for quick checks
    "tsm8": dict(L=(8, 8, 8, 8), kappa=0.161, mu=0.003, n_hp=4, n_lp=28, batch=16,
                 lp_prec="f16", hp_inner="f32", tol_lp=1e-2, tol_hp=1e-9, gauge_seed=1237,
                 seed=20140126, schur=True, delta=3e-5, recon=0, overlap=False, hp_loops="ff", hp_ru="f64"),
}

FP32_LANES_PER_SM = 128    # FP32 FMA lanes per SM (4 partitions x 32)
PREC_BYTES = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2, "ff": 8}
METRIC = "Dslash HBM GB/s and % roofline; TSM loop sec/source at fixed error vs FP64 CG"


def workload_name(c):
    X, Y, Z, T = c["L"]
    return ("TSM loops %dx%dx%dx%d kappa=%g mu=%g: %d LP (%s, |r|<=%g) + %d HP (mixed %s/FP64, %s residuals, "
            "|r|<=%g, delta=%g%s), batches of %d, %s CG, local+oneD x (one-end, generalised one-end)" % (
                X, Y, Z, T, c["kappa"], c["mu"], c["n_lp"] + c["n_hp"], c["lp_prec"], c["tol_lp"],
                c["n_hp"], c["hp_inner"], "float-float" if c.get("hp_ru") == "ff" else "FP64",
                c["tol_hp"], c["delta"],
                ", on a second stream" if c.get("overlap") else "", c["batch"],
                "even/odd-preconditioned" if c["schur"] else "unpreconditioned"))


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.path = None

    @staticmethod
    def device_id():
        """nvidia-smi's id of this process's GPU: its UUID (CUDA ordinals differ from
        nvidia-smi's indices when CUDA_VISIBLE_DEVICES remaps them)."""
        import torch
        dev = torch.cuda.current_device()
        try:
            uid = str(torch.cuda.get_device_properties(dev).uuid)
            if uid and uid != "None":
                return uid if uid.startswith(("GPU-", "MIG-")) else "GPU-" + uid
        except (AttributeError, RuntimeError):
            pass
        vis = [v.strip() for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
        return vis[dev] if dev < len(vis) else str(dev)

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", self.device_id()],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
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
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons, "samples": len(rows)}


def _log(msg):
    if int(os.environ.get("RANK", "0")) == 0:
        sys.stderr.write("[bench %.1fs] %s\n" % (time.perf_counter() - _T0, msg))
        sys.stderr.flush()


_T0 = time.perf_counter()


# ----------------------------------------------------------------- ours
def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        return dist, rank, world
    return None, 0, 1


def _max_over_ranks(dist, v):
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(dist):
    if dist is not None:
        dist.barrier()


# ncu DRAM traffic per algorithmic byte, per Dslash kernel class: the
# committed summary and the sources its capture was taken from
TRAFFIC_FILES = {"dslash.f16il": ("dslash_il_traffic.txt", ("dslash_il.cu", "il_core.cuh", "tm_core.cuh")),
                 "dslash.bf16il": ("dslash_il_traffic.txt", ("dslash_il.cu", "il_core.cuh", "tm_core.cuh")),
                 "dslash.f16": ("dslash_traffic.txt", ("dslash.cuh", "tm_core.cuh")),
                 "dslash.bf16": ("dslash_traffic.txt", ("dslash.cuh", "tm_core.cuh"))}


def _traffic_per_launch(alg_bytes, kernel="dslash.f16.out"):
    """DRAM bytes per launch of a Dslash kernel class: the ncu-measured traffic
    per algorithmic byte (profiles/<file>) times this launch's algorithmic
    bytes; None if there is no capture for the class or its kernel sources
    changed since the capture."""
    import hashlib
    entry = TRAFFIC_FILES.get(kernel.rsplit(".", 1)[0])
    if entry is None:
        return None
    path = os.path.join(ROOT, "profiles", entry[0])
    if not os.path.exists(path):
        return None
    kv = {}
    with open(path) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
    csrc = os.path.join(ROOT, "paper_1401_6749_gb300", "csrc")
    src = b"".join(open(os.path.join(csrc, n), "rb").read() for n in entry[1])
    if hashlib.sha256(src).hexdigest() != kv.get("kernel_sources_sha256"):
        return None
    return int(round(float(kv["traffic_per_algorithmic_byte"]) * alg_bytes))


def _tuned_shapes(tl, L):
    """The autotuner's launch shapes for this lattice's half volume:
    "<prec>.<out|resid>.<parity>.<n systems>" -> "<systems per thread>[p]x<threads per block>"
    (p: packed FP32x2 arithmetic)."""
    vh = L[0] * L[1] * L[2] * L[3] // 2
    pn = {0: "f64", 1: "f32", 2: "f16", 3: "bf16", 4: "ff"}
    out = {}
    for key, nr, bx, pk in tl.tm_tune_entries():
        if key["half_volume"] != vh:
            continue
        name = "%s%s.%s.%s.n%d" % (pn[key["prec"]], ".dag" if key["dagger"] else "",
                                   "resid" if key["epilogue"] == 2 else "out",
                                   {-1: "both", 0: "even", 1: "odd"}[key["parity"]], key["nrhs"])
        out[name] = "%d%sx%d" % (nr, "p" if pk else "", bx)
    return out


def _dslash_alone(tl, op, L, prec, n, recon, warmup=5, reps=20, il=False):
    """tm_dslash (M on both parities) of n Z4 fields on the workload's operator,
    timed with CUDA events after warm-up; algorithmic bytes per launch are
    n x (in + out) spinors plus the links once.  il: the same fields in the
    system-interleaved layout through tm_dslash_il (tensor cores)."""
    import torch
    V = L[0] * L[1] * L[2] * L[3]
    fin = tl.empty_field(L, prec, n)
    fout = tl.empty_field(L, prec, n)
    tl.z4_noise(L, fin, prec, 7, 0, n)
    apply = lambda: tl.tm_dslash(op, fout, fin, n, prec=prec)
    if il:
        fin_il = tl.empty_field_il(L, n)
        fout_il = tl.empty_field_il(L, n)
        tl.tm_spinor_to_il(L, fin_il, fin, prec, n)
        del fin, fout
        apply = lambda: tl.tm_dslash_il(op, fout_il, fin_il, n, prec=prec)
    for _ in range(warmup):
        apply()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        apply()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    esz = tl.ELEM_SIZE[prec]
    nbytes = n * 2 * 24 * esz * V + 4 * tl.link_reals(recon, prec) * esz * V
    peak, src = _peaks()
    gbs = nbytes / (ms * 1e-3) / 1e9
    return {"nrhs": n, "ms_per_launch": round(ms, 4), "GBps": round(gbs, 1), "frac_of_hbm": round(gbs / peak, 4),
            "link_reals": tl.link_reals(recon, prec), "peak_source": src}


def _observables(pipe, c):
    """Per-source values of three volume-summed loops (sigma-term, g_A and
    Fig. 1 operator analogues) for the HP and LP sets, on the host."""
    import numpy as np
    T = c["L"][3]
    nu = 2 * c["kappa"] * c["mu"]
    out = {}

    def cplx(t):
        return t.cpu().numpy().view(np.complex128).reshape(t.shape[0], -1, T)

    lp = {k: cplx(v) for k, v in pipe.lp_loops.items()}
    hp = {k: cplx(v) for k, v in pipe.hp_loops.items()}
    # sigma-term analogue: Gamma = 1, one-end trick (-2 i nu);  g_A analogue:
    # Gamma_11 = g1 g2 g4 = g3 g5, generalised trick (2);  Fig. 1: i psibar g3 D3 psi,
    # generalised trick, mu = z, Gamma_4 = g3.
    sel = {"sigma": ("local_vv", 0, -2j * nu), "gA": ("local_gen", 11, 2.0),
           "g3D3": ("oneD_gen", 2 * 16 + 4, 2.0j)}
    for name, (k, row, sc) in sel.items():
        out[name] = (sc * hp[k][:, row, :].sum(axis=1), sc * lp[k][:, row, :].sum(axis=1))
    return out


def _tsm_efficiency(obs_step, obs_side, c, t_step, t_plain_src, phase):
    """The paper's efficiency ratios of the TSM (Sec. 4, Table tab:TSM and
    Table compRatios) for three volume-summed observables.

    TSM error of the step:  err^2 = Var(hp - lp) / N_HP + Var(lp) / N_LP (Eq. 4);
    plain estimator: N_plain = N_HP + N_LP high-precision sources (as many
    stochastic sources as the step), err^2 = Var(hp) / N_plain, cost
    N_plain x t_plain (single-system FP64 CG on this GPU with the same
    contractions).  R_E = err_TSM / err_plain, R_C = t_step / (N_plain t_plain),
    R_C R_E^2 and its inverse (the equal-error speedup) do not depend on
    N_plain.  The variances come from the step's N_HP paired (HP, LP) sources
    plus the side run's paired sources (Var(hp), Var(hp - lp)) and from every
    LP value (Var(lp)); errors by jackknife over the paired sources.
    R_HP/LP (Sec. 4): time of one HP source (solve + contractions) over that
    of one LP source, with the local loops only and with the one-derivative
    loops as well, from the phase times of one step."""
    import numpy as np
    n_hp, n_lp = c["n_hp"], c["n_lp"]
    n_plain = n_hp + n_lp
    out = {"definition": "R_E = err_TSM / err_plain, R_C = cost_TSM / cost_plain with N_plain = N_HP + N_LP "
                         "plain FP64-CG sources; R_C R_E^2 independent of N_plain; jackknife errors over "
                         "paired (HP, LP) sources",
           "n_plain": n_plain, "observables": {}}
    for name in obs_step:
        hp = np.concatenate([obs_step[name][0], obs_side[name][0]])
        lp_pair = np.concatenate([obs_step[name][1][:n_hp], obs_side[name][1]])
        lp_rest = obs_step[name][1][n_hp:]
        npair = hp.size

        def ratios(keep):
            h, lpp = hp[keep], lp_pair[keep]
            var_d = (h - lpp).var(ddof=1)
            var_lp = np.concatenate([lpp, lp_rest]).var(ddof=1)
            var_plain = h.var(ddof=1)
            err2_tsm = var_d / n_hp + var_lp / n_lp
            err2_plain = var_plain / n_plain
            r_e = float(np.sqrt(err2_tsm / err2_plain))
            r_c = float(t_step / (n_plain * t_plain_src))
            return r_e, r_c, r_c * r_e ** 2
        r_e, r_c, prod = ratios(np.ones(npair, bool))
        jk = np.array([ratios(np.arange(npair) != i) for i in range(npair)])
        jerr = np.sqrt((npair - 1) / npair * ((jk - jk.mean(axis=0)) ** 2).sum(axis=0))
        out["observables"][name] = {"R_E": round(r_e, 4), "R_E_err": round(float(jerr[0]), 4),
                                    "R_C": round(r_c, 5), "R_C_R_E2": round(prod, 5),
                                    "R_C_R_E2_err": round(float(jerr[2]), 5),
                                    "equal_error_speedup": round(1.0 / prod, 2) if prod > 0 else None,
                                    "paired_sources": int(npair), "lp_values": int(npair + lp_rest.size)}
    if phase:
        t_hp = {k: v / n_hp for k, v in phase["hp"].items()}
        t_lp = {k: v / (n_hp + n_lp) for k, v in phase["lp"].items()}
        out["R_HP_LP"] = {
            "local": round((t_hp["solve"] + t_hp["local"]) / (t_lp["solve"] + t_lp["local"]), 2),
            "with_one_derivative": round(sum(t_hp.values()) / sum(t_lp.values()), 2),
            "ms_per_source": {"hp": {k: round(v, 3) for k, v in t_hp.items()},
                              "lp": {k: round(v, 4) for k, v in t_lp.items()}}}
    out["paper_context"] = ("paper (unnamed GPUs, real N_f=2+1+1 ensemble, one-end trick): R_C R_E^2 light "
                            "0.73 (sigma-term) / 0.15 (g_A); R_HP/LP light ~26.7 local, ~10 with one-derivative")
    return out


# twisted masses standing in for the paper's three sectors (Sec. 3: strange
# and charm near their physical values; the ensemble's own values are not
# given): the light mass of the workload, and strange / charm masses about
# 13 and 170 times heavier in lattice units
SECTOR_MU = {"strange": 0.04, "charm": 0.5}


def _efficiency_of(tl, TsmPipeline, op, pipe, c, ms, dist, rank, world, n_src, mk):
    """Plain FP64 CG time per source on op, phase times of one step, a side run
    of paired sources, and the efficiency ratios (_tsm_efficiency) of the
    pipeline `pipe` whose step took `ms` milliseconds."""
    import numpy as np
    import torch
    L = c["L"]
    n_plain = 2
    eta = tl.empty_field(L, tl.F64, 1)
    x = tl.empty_field(L, tl.F64, 1)
    w = tl.empty_field(L, tl.F64, 1)
    g5w = tl.empty_field(L, tl.F64, 1)
    T = L[3]
    loc = torch.empty(32 * T, dtype=torch.float64, device="cuda")
    oned = torch.empty(128 * T, dtype=torch.float64, device="cuda")
    prm = tl.cg_params(c["tol_hp"], 20000, tl.CG_PLAIN, prec=tl.F64, check_every=8, schur=c["schur"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for j in range(n_plain):
        tl.z4_noise(L, eta, tl.F64, c["seed"], rank * n_src + j, 1)
        tl.tm_cg_solve(op, x, eta, 1, prm)
        tl.tm_dslash(op, w, x, 1, mu_zero=True, prec=tl.F64)
        tl.tm_gamma5(L, g5w, w, tl.F64, 1)
        for left, right, mode in ((x, x, tl.LOOP_VV), (x, g5w, tl.LOOP_GEN)):
            tl.loop_contract_local(L, left, right, tl.F64, 1, mode, loc)
            tl.loop_contract_oneD(op, left, right, tl.F64, 1, mode, oned)
    torch.cuda.synchronize()
    t_plain = (time.perf_counter() - t0) / n_plain
    _log("plain FP64 CG (mu %g): %.3f s/source" % (c["mu"], t_plain))
    del eta, x, w, g5w
    # phase times of one step (solve / local loops / one-derivative loops of
    # the LP and HP sets) and the variances from a side run of paired (HP, LP)
    # sources beyond the step's, both outside the timed region
    pt = mk(op, timing=True)
    pt.run(dist)
    phase = pt.phase_ms()
    del pt
    obs_step = _observables(pipe, c)
    n_side = 32
    side = TsmPipeline(op, n_side, 0, batch=c["n_hp"], lp_prec=tl.PREC[c["lp_prec"]],
                       hp_inner=tl.PREC[c["hp_inner"]], tol_lp=c["tol_lp"], tol_hp=c["tol_hp"],
                       seed=c["seed"], first_src=world * n_src + rank * n_side, schur=c["schur"],
                       delta=c["delta"], hp_loop_prec=tl.PREC[c["hp_loops"]], hp_ru_prec=tl.PREC[c["hp_ru"]])
    side.run_sources()
    side_ok = all(s["status"] == 0 for s in side.stats_hp + side.stats_lp)
    obs_side = _observables(side, dict(c, n_hp=n_side))
    eff = _tsm_efficiency(obs_step, obs_side, c, ms * 1e-3, t_plain, phase)
    eff["side_run_converged"] = side_ok
    eff["fp64_cg_plain_s_per_source"] = round(t_plain, 4)
    lp_it = [q["iters"] for q in pipe.stats_lp]
    hp_it = [q["iters"] for q in pipe.stats_hp]
    eff["field_note"] = ("synthetic smooth gauge field: the solves converge in few iterations (LP mean %.1f, HP "
                         "mean %.1f, even/odd), so the step is dominated by per-source fixed costs (contractions, "
                         "D_W) rather than by the solves, unlike a real ensemble" % (
                             float(np.mean(lp_it)) if lp_it else 0.0, float(np.mean(hp_it)) if hp_it else 0.0))
    return eff, t_plain


def run_ours(args):
    import numpy as np
    import torch
    dist, rank, world = _dist()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    import __graft_entry__
    # rank 0 builds the library; the other ranks wait, then find it up to date
    # (the build also serialises concurrent callers on a lock file)
    if rank == 0:
        __graft_entry__.build()
    _barrier(dist)
    if rank != 0:
        __graft_entry__.build()
    from paper_1401_6749_gb300 import synth
    from paper_1401_6749_gb300 import tmloops as tl
    from paper_1401_6749_gb300.tsm_pipeline import TsmPipeline

    c = CONFIGS[args.config]
    L = c["L"]
    V = int(np.prod(L))
    U = synth.gauge_field(L, c["gauge_seed"], device="cuda")
    U_host = torch.from_numpy(U.view(np.float64)).pin_memory()
    U_dev = U_host.cuda()
    del U
    op = tl.Operator(L, c["kappa"], c["mu"], U_dev, recon=c["recon"])
    n_src = c["n_hp"] + c["n_lp"]
    mk = lambda o, **kw: TsmPipeline(o, c["n_hp"], c["n_lp"], batch=c["batch"], lp_prec=tl.PREC[c["lp_prec"]],
                               hp_inner=tl.PREC[c["hp_inner"]], tol_lp=c["tol_lp"], tol_hp=c["tol_hp"],
                               seed=c["seed"], first_src=rank * n_src, schur=c["schur"],
                               delta=c["delta"], overlap=c["overlap"], hp_loop_prec=tl.PREC[c["hp_loops"]],
                               hp_ru_prec=tl.PREC[c["hp_ru"]], **kw)
    pipe = mk(op)
    _log("inputs ready")
    for _ in range(args.warmup):
        pipe.run(dist)
    torch.cuda.synchronize()
    _log("warm-up done: LP iters %s, HP iters %s" % ([s["iters"] for s in pipe.stats_lp][:16],
                                                     [s["iters"] for s in pipe.stats_hp]))

    # ---- timed region: inputs resident in HBM
    clocks = ClockSampler()
    clocks.start()
    tl.tm_trace_reset()
    tl.tm_trace_enable(True)
    launches0 = tl.tm_launch_count()
    _barrier(dist)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        res = pipe.run(dist)
    ev1.record()
    torch.cuda.synchronize()
    _barrier(dist)
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = (tl.tm_launch_count() - launches0) // args.steps
    tl.tm_trace_enable(False)
    clk = clocks.stop()
    classes = {}
    precs = ("f64", "f32", "f16", "bf16", "ff")
    names = ["dslash.%s.%s" % (p, e) for p in precs + ("f16il", "bf16il") for e in ("out", "cgupd", "resid")]
    names += ["%s.%s" % (k, p) for k in ("local", "oneD") for p in precs + ("f16il", "bf16il")]
    names += ["blas.xpay", "z4_noise", "cg.graph"]
    flops = {}
    for name in names:
        n, tms, nbytes = tl.tm_trace_read(name)
        if n:
            classes[name] = (n / args.steps, tms / args.steps, nbytes / args.steps)
            flops[name] = tl.tm_trace_read_flops(name) / args.steps
    tl.tm_trace_reset()
    ms = _max_over_ranks(dist, ms)
    _log("timed: %.3f ms/step, %d launches/step, classes %s" % (ms, launches, classes))

    # ---- roofline of the dominant Dslash class (by device time): algorithmic
    # bytes recorded per launch by the library (active systems only), device
    # time from CUDA events on the launch stream
    peak, peak_src = _peaks()
    kernels = {}
    for name, (n, tms, nbytes) in classes.items():
        kernels[name] = {"launches": round(n, 1), "ms": round(tms, 3), "share_of_step": round(tms / ms, 4),
                         "GBps": round(nbytes / (tms * 1e-3) / 1e9, 1) if tms > 0 else None}
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    n_dom, t_dom, b_dom = classes[dom]
    ach = kernels[dom]["GBps"]
    traffic = _traffic_per_launch(b_dom / n_dom, dom) if dom.startswith("dslash.") else None
    hbm_view = {"achieved": ach, "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
                "peak_source": peak_src}
    flops_dom = flops.get(dom, 0.0)
    if dom.startswith(("dslash.f16.", "dslash.bf16.")) and flops_dom > 0:
        # the 16-bit Dslash is bound by FP32 instruction issue (ncu: issue 78%,
        # FMA pipe 60%, DRAM 27%): roofline against the FP32 peak derived from
        # the unit counts and the SM clock sampled during the timed region
        sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
        n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        alu_peak = n_sm * FP32_LANES_PER_SM * 2.0 * sm_mhz * 1e6 / 1e12
        tflops = flops_dom / (t_dom * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": round(tflops, 2), "peak": round(alu_peak, 2), "unit": "TFLOP/s",
                    "frac": round(tflops / alu_peak, 4), "traffic": traffic, "kernel": dom,
                    "peak_source": "derived: %d SMs x 128 FP32 lanes x 2 flop x %.0f MHz (sampled)"
                                   % (n_sm, sm_mhz),
                    "algorithmic_flops_per_launch": round(flops_dom / n_dom),
                    "algorithmic_bytes_per_launch": round(b_dom / n_dom), "hbm": hbm_view}
    else:
        roofline = dict(bound="hbm", **{k: v for k, v in hbm_view.items()}, traffic=traffic, kernel=dom,
                        algorithmic_bytes_per_launch=round(b_dom / n_dom))

    # ---- the Dslash alone on the workload's lattice: FP32 with one system
    # (bandwidth bound, the HBM roofline target) and FP16 with a batch of 16
    dslash_alone = {"f32": _dslash_alone(tl, op, L, tl.F32, 1, c["recon"]),
                    "f16": _dslash_alone(tl, op, L, tl.F16, c["batch"], c["recon"]),
                    "f16il": _dslash_alone(tl, op, L, tl.F16, c["batch"], c["recon"], il=True)}

    # ---- correctness/quality summary of the last step
    it_lp = [s["iters"] for s in pipe.stats_lp]
    it_hp = [s["iters"] for s in pipe.stats_hp]
    ok = all(s["status"] == 0 for s in pipe.stats_lp + pipe.stats_hp)

    # ---- plain single-RHS FP64 CG on the same GPU (equal-error baseline),
    # the paper's efficiency ratios, and the same for the heavier sectors
    t_plain = None
    efficiency = None
    sectors = None
    if not args.no_baseline:
        efficiency, t_plain = _efficiency_of(tl, TsmPipeline, op, pipe, c, ms, dist, rank, world, n_src, mk)
        sectors = {"light": dict(mu=c["mu"], step_ms=round(ms, 3), **efficiency)}
        for name, mu_s in SECTOR_MU.items():
            cs = dict(c, mu=mu_s)
            op_s = tl.Operator(L, c["kappa"], mu_s, U_dev, recon=c["recon"])
            mk_s = lambda o, **kw: TsmPipeline(o, cs["n_hp"], cs["n_lp"], batch=cs["batch"],
                                               lp_prec=tl.PREC[cs["lp_prec"]], hp_inner=tl.PREC[cs["hp_inner"]],
                                               tol_lp=cs["tol_lp"], tol_hp=cs["tol_hp"], seed=cs["seed"],
                                               first_src=rank * n_src, schur=cs["schur"], delta=cs["delta"],
                                               hp_loop_prec=tl.PREC[cs["hp_loops"]],
                                               hp_ru_prec=tl.PREC[cs["hp_ru"]], **kw)
            p_s = mk_s(op_s)
            p_s.run(dist)  # warm-up
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            p_s.run(dist)
            e1.record()
            torch.cuda.synchronize()
            ms_s = _max_over_ranks(dist, e0.elapsed_time(e1))
            eff_s, _ = _efficiency_of(tl, TsmPipeline, op_s, p_s, cs, ms_s, dist, rank, world, n_src, mk_s)
            sectors[name] = dict(mu=mu_s, step_ms=round(ms_s, 3),
                                 lp_iters_mean=round(float(np.mean([q["iters"] for q in p_s.stats_lp])), 2),
                                 hp_iters_mean=round(float(np.mean([q["iters"] for q in p_s.stats_hp])), 2),
                                 **eff_s)
            _log("sector %s (mu %g): %.3f ms/step" % (name, mu_s, ms_s))
            del p_s
            op_s.close()

    # ---- end to end through host buffers: H2D gauge field, operator set-up,
    # the full step, D2H of the combined loops, every step
    e2e = None
    if not args.no_e2e:
        res_bytes = sum(2 * m.numel() * 8 for m, _ in res.values())
        host_out = [torch.empty(m.numel() * 2, dtype=torch.float64).pin_memory() for m, _ in res.values()]

        def e2e_step():
            # the operator reads the gauge field from pinned host memory itself
            # (one pass of the SMs over the host link), every step
            op2 = tl.Operator(L, c["kappa"], c["mu"], U_host, recon=c["recon"])
            p2 = mk(op2)
            r2 = p2.run(dist)
            for h, (m, e) in zip(host_out, r2.values()):
                h[: m.numel()].copy_(m, non_blocking=True)
                h[m.numel():].copy_(e, non_blocking=True)
            torch.cuda.synchronize()
            del p2
            op2.close()

        # one untimed step: the library's memory pool grows to hold a second
        # operator beside the resident one; later steps reuse that memory
        e2e_step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        _barrier(dist)
        e0.record()
        for _ in range(args.steps):
            e2e_step()
        e1.record()
        torch.cuda.synchronize()
        ems = _max_over_ranks(dist, e0.elapsed_time(e1) / args.steps)
        _log("e2e: %.3f ms/step" % ems)
        e2e = {"value": round(ems * 1e-3 / (world * n_src), 6), "unit": "s/source",
               "h2d_bytes_per_step": int(U_host.numel() * 8), "d2h_bytes_per_step": int(res_bytes)}

    # ---- CPU baseline: the oracle on the host cores (rank 0, N = 1).  The
    # oracle's CG is unpreconditioned: its iteration counts per source are
    # those of the unpreconditioned solver, measured here on one LP and one HP
    # source (equal in exact arithmetic)
    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        e1 = tl.empty_field(L, tl.PREC[c["lp_prec"]], 1)
        x1 = tl.empty_field(L, tl.PREC[c["lp_prec"]], 1)
        tl.z4_noise(L, e1, tl.PREC[c["lp_prec"]], c["seed"], 0, 1)
        _, s_lp = tl.tm_cg_solve(op, x1, e1, 1, tl.cg_params(c["tol_lp"], 20000, tl.CG_PLAIN,
                                                             prec=tl.PREC[c["lp_prec"]]))
        e2 = tl.empty_field(L, tl.F64, 1)
        x2 = tl.empty_field(L, tl.F64, 1)
        tl.z4_noise(L, e2, tl.F64, c["seed"], 0, 1)
        _, s_hp = tl.tm_cg_solve(op, x2, e2, 1, tl.cg_params(c["tol_hp"], 20000, tl.CG_MIXED,
                                                             inner_prec=tl.F32, delta=0.1))
        n_lp_all = c["n_hp"] + c["n_lp"]
        cpu = cpu_baseline(c, [s_lp[0]["iters"]] * n_lp_all, [s_hp[0]["iters"]] * c["n_hp"])

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(ms * 1e-3 / (world * n_src), 6), "unit": "s/source",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f16",
            "dtype_detail": ("LP solves f16 (f32 arithmetic); HP solves f32 inner, reliable-update and final "
                             "residuals " + ("float-float (~48-bit)" if c["hp_ru"] == "ff" else "f64") +
                             ", f64 solution accumulation and dot products; HP loops (D_W s and contractions) "
                             + ("float-float (~48-bit) arithmetic on the f64 solutions" if c["hp_loops"] == "ff"
                                else "f64") + "; loop sums f64"),
            "data": "synthetic: smooth random SU(3) links U = exp(0.3 i H), Z4 sources",
            "config": {"workload": workload_name(c), "lattice": list(L), "n_sources": n_src,
                       "l2": "inputs larger than L2 (fields of 100-400 MB each)",
                       "parallelism": "sources sharded over %d rank(s); per-source loops all-gathered "
                                      "for the global TSM combination" % world},
            "roofline": roofline, "kernels": kernels,
            "gpu_launches": int(launches),
            "e2e": e2e, "cpu_baseline": cpu, "clocks": clk,
            "solver": {"lp_iters_mean": round(float(np.mean(it_lp)), 2), "lp_iters_max": int(max(it_lp)),
                       "hp_iters": it_hp, "hp_reliable_updates": [s["reliable_updates"] for s in pipe.stats_hp],
                       "hp_true_res_max": max(s["true_res"] for s in pipe.stats_hp) if pipe.stats_hp else None,
                       "all_converged": ok},
            "fp64_cg_plain_s_per_source": round(t_plain, 4) if t_plain else None,
            "tsm_efficiency": efficiency,
            "sectors": sectors,
            "dslash_shapes": _tuned_shapes(tl, L),
            "dslash_alone": dslash_alone,
        }
        print(json.dumps(line), flush=True)
    op.close()
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------- standalone Dslash
def run_dslash(args):
    """Time tm_dslash alone: M applied to nrhs Z4 fields (seed 7), the
    per-launch time averaged over --steps launches after --warmup launches.
    Algorithmic bytes per launch: nrhs x (in + out spinor) + the links once."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1401_6749_gb300 import synth
    from paper_1401_6749_gb300 import tmloops as tl
    L = tuple(int(v) for v in args.lattice.split(","))
    prec = tl.PREC[args.prec]
    n = args.nrhs
    V = int(np.prod(L))
    U = synth.gauge_field(L, 1234, device="cuda")
    op = tl.Operator(L, 0.161, 0.003, torch.from_numpy(U.view(np.float64)).cuda(), recon=args.recon)
    del U
    fin = tl.empty_field(L, prec, n)
    fout = tl.empty_field(L, prec, n)
    tl.z4_noise(L, fin, prec, 7, 0, n)
    apply = lambda: tl.tm_dslash(op, fout, fin, n, prec=prec)
    if args.layout == "il":
        # the same fields in the system-interleaved layout, tensor-core kernel
        fin_il = tl.empty_field_il(L, n)
        fout_il = tl.empty_field_il(L, n)
        tl.tm_spinor_to_il(L, fin_il, fin, prec, n)
        del fin, fout
        apply = lambda: tl.tm_dslash_il(op, fout_il, fin_il, n, prec=prec)
    for _ in range(args.warmup):
        apply()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        apply()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    esz = tl.ELEM_SIZE[prec]
    link_reals = tl.link_reals(args.recon, prec)
    nbytes = n * 2 * 24 * esz * V + 4 * link_reals * esz * V
    peak, src = _peaks()
    gbs = nbytes / (ms * 1e-3) / 1e9
    print(json.dumps({"mode": "dslash", "layout": args.layout, "lattice": list(L), "nrhs": n, "prec": args.prec,
                      "recon": link_reals, "ms_per_launch": round(ms, 4), "bytes_per_launch": nbytes,
                      "GBps": round(gbs, 1), "frac_of_hbm": round(gbs / peak, 4), "peak_source": src,
                      "l2": "in+out fields %.0f MB" % (2 * n * 24 * esz * V / 1e6)}), flush=True)
    op.close()


def run_contract(args):
    """Time the loop contractions alone on nrhs Z4 fields (seeds 7 and 8):
    loop_contract_local and loop_contract_oneD (one-end mode), per launch
    averaged over --steps launches after --warmup.  Algorithmic bytes per
    launch: nrhs x 2 spinors (+ the links once for oneD); useful flops per site
    and system: 384 (local, the 4 x 4 spin matrix) and 4224 (oneD: per mu two
    link products of a 4-spinor and the spin outer products, the time
    direction with two of each)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1401_6749_gb300 import synth
    from paper_1401_6749_gb300 import tmloops as tl
    L = tuple(int(v) for v in args.lattice.split(","))
    prec = tl.PREC[args.prec]
    n = args.nrhs
    V = int(np.prod(L))
    U = synth.gauge_field(L, 1234, device="cuda")
    op = tl.Operator(L, 0.161, 0.003, torch.from_numpy(U.view(np.float64)).cuda(), recon=args.recon)
    del U
    a = tl.empty_field(L, prec, n)
    b = tl.empty_field(L, prec, n)
    tl.z4_noise(L, a, prec, 7, 0, n)
    tl.z4_noise(L, b, prec, 8, 0, n)
    T = L[3]
    out = torch.empty(n * 64 * T * 2, dtype=torch.float64, device="cuda")
    if args.layout == "il":
        # the same fields in the system-interleaved layout (tensor-core oneD)
        ai, bi = tl.empty_field_il(L, n), tl.empty_field_il(L, n)
        tl.tm_spinor_to_il(L, ai, a, prec, n)
        tl.tm_spinor_to_il(L, bi, b, prec, n)
        del a, b
        jobs = {"local": (lambda: tl.loop_contract_local_il(L, ai, bi, prec, n, tl.LOOP_VV, out), 384.0, False),
                "oneD": (lambda: tl.loop_contract_oneD_il(op, ai, bi, prec, n, tl.LOOP_VV, out), 4224.0, True)}
    else:
        jobs = {"local": (lambda: tl.loop_contract_local(L, a, b, prec, n, tl.LOOP_VV, out), 384.0, False),
                "oneD": (lambda: tl.loop_contract_oneD(op, a, b, prec, n, tl.LOOP_VV, out), 4224.0, True)}
    esz = tl.ELEM_SIZE[prec]
    link_reals = tl.link_reals(args.recon, prec)
    peak, src = _peaks()
    res = {}
    for name, (fn, flops, links) in jobs.items():
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        nbytes = n * 2 * 24 * esz * V + (4 * link_reals * esz * V if links else 0)
        res[name] = {"ms_per_launch": round(ms, 4), "GBps": round(nbytes / (ms * 1e-3) / 1e9, 1),
                     "frac_of_hbm": round(nbytes / (ms * 1e-3) / 1e9 / peak, 4),
                     "TFLOPs": round(flops * V * n / (ms * 1e-3) / 1e12, 2)}
    if args.layout == "il":
        tl.tm_op_check(op)
    print(json.dumps({"mode": "contract", "layout": args.layout, "lattice": list(L), "nrhs": n, "prec": args.prec,
                      "recon": link_reals, "peak_source": src, "kernels": res}), flush=True)
    op.close()


# ------------------------------------------------------- widened rows
def run_next(args):
    """Time the widened rows on 16 systems at the workload's lattice: the HPE
    remainder (BH)^4 s (Sec. 2.4), time-diluted Z4 sources (Sec. 2.3) and
    momentum-projected local loops with 8 momenta; prints one JSON line."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1401_6749_gb300 import synth
    from paper_1401_6749_gb300 import tmloops as tl
    c = CONFIGS[args.config]
    L = c["L"]
    V = int(np.prod(L))
    n = 16
    prec = tl.PREC[c["lp_prec"]]
    esz = tl.ELEM_SIZE[prec]
    U = synth.gauge_field(L, c["gauge_seed"], device="cuda")
    op = tl.Operator(L, c["kappa"], c["mu"], torch.from_numpy(U.view(np.float64)).cuda(), recon=c["recon"])
    del U
    a = tl.empty_field(L, prec, n)
    b = tl.empty_field(L, prec, n)
    tl.z4_noise(L, a, prec, 7, 0, n)
    moms = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1)]
    T = L[3]
    out = torch.empty(n * len(moms) * 16 * T * 2, dtype=torch.float64, device="cuda")
    jobs = {
        "hpe_BH4": lambda: tl.tm_hpe_apply(op, b, a, n, 4, prec),
        "z4_time_diluted": lambda: tl.z4_noise_diluted(L, b, prec, 7, 0, n, 3, 8),
        "local_mom8": lambda: tl.loop_contract_local_mom(L, a, b, prec, n, tl.LOOP_STD, moms, out),
    }
    res = {}
    for name, fn in jobs.items():
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        res[name] = {"ms": round(e0.elapsed_time(e1) / args.steps, 4)}
    spin = 24 * esz * V
    link = 4 * tl.link_reals(c["recon"], prec) * esz * V
    nbytes = {"hpe_BH4": 4 * (n * 2 * spin + link), "z4_time_diluted": n * spin, "local_mom8": n * 2 * spin}
    peak, src = _peaks()
    for k, v in res.items():
        gbs = nbytes[k] / (v["ms"] * 1e-3) / 1e9
        v["GBps"] = round(gbs, 1)
        v["frac_of_hbm"] = round(gbs / peak, 4)
    t0 = time.perf_counter()
    tl.tm_hpe_exact(L, c["kappa"], c["mu"])
    res["hpe_exact_terms_host_ms"] = round((time.perf_counter() - t0) * 1e3, 3)
    print(json.dumps({"mode": "next", "lattice": list(L), "nrhs": n, "prec": c["lp_prec"],
                      "peak_source": src, "kernels": res}), flush=True)
    op.close()


def run_solvers(args):
    """Time whole solves, graph replay against eager launches:
      * 24^3 x 48, kappa = 0.161, mu = 0.004: 12 and 24 Z4 sources in one
        batched mixed-precision solve (FP32 iteration, FP64 reliable updates,
        tol 1e-10, even/odd);
      * the uneven batch 8^4 / 12^4 / 16^3 x 32 / 24^3 x 48 (kappa 0.155 ..
        0.162, mu 0.01 .. 0.003, 4 / 8 / 16 / 32 sources): the TSM solves (FP16
        to 1e-2 and mixed to 1e-9) of the four lattices one after the other,
        as one group, and as one group replayed as graphs.
    Prints one JSON line with ms per solve (median over --steps)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1401_6749_gb300 import synth
    from paper_1401_6749_gb300 import tmloops as tl

    def make_op(L, k, m, seed):
        U = synth.gauge_field(L, seed, device="cuda")
        return tl.Operator(L, k, m, torch.from_numpy(U.view(np.float64)).cuda(), recon=0)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append((time.perf_counter() - t0) * 1e3)
        return round(float(np.median(ts)), 3)

    res = {}
    L = (24, 24, 24, 48)
    op = make_op(L, 0.161, 0.004, 1236)
    for n in (12, 24):
        eta = tl.empty_field(L, tl.F64, n)
        tl.z4_noise(L, eta, tl.F64, 20140126, 0, n)
        x = tl.empty_field(L, tl.F64, n)
        for graph in (False, True):
            prm = tl.cg_params(1e-10, 20000, tl.CG_MIXED, inner_prec=tl.F32, delta=1e-5, check_every=4,
                               schur=True, graph=graph)
            res[f"24x48_mixed_n{n}_{'graph' if graph else 'eager'}_ms"] = timed(
                lambda: tl.tm_cg_solve(op, x, eta, n, prm))
        del eta, x
    op.close()
    ragged = [((8, 8, 8, 8), 0.155, 0.01, 4), ((12, 12, 12, 12), 0.158, 0.007, 8),
              ((16, 16, 16, 32), 0.160, 0.005, 16), ((24, 24, 24, 48), 0.162, 0.003, 32)]
    ops = [make_op(Lr, k, m, 1238) for Lr, k, m, _ in ragged]
    ns = [n for *_, n in ragged]
    for name, fp, base in (("lp", tl.F16, dict(tol=1e-2, mode=tl.CG_PLAIN, prec=tl.F16, check_every=2)),
                           ("hp", tl.F64, dict(tol=1e-9, mode=tl.CG_MIXED, inner_prec=tl.F32, delta=3e-5,
                                               check_every=4))):
        etas = [tl.empty_field(Lr, fp, n) for (Lr, *_), n in zip(ragged, ns)]
        xs = [tl.empty_field(Lr, fp, n) for (Lr, *_), n in zip(ragged, ns)]
        for (Lr, *_), e, n in zip(ragged, etas, ns):
            tl.z4_noise(Lr, e, fp, 20140126, 0, n)
        kw = dict(base)
        tol = kw.pop("tol")
        eager = tl.cg_params(tol, 20000, schur=True, graph=False, **kw)
        graph = tl.cg_params(tol, 20000, schur=True, graph=True, **kw)

        def seq(prm):
            for o, x, e, n in zip(ops, xs, etas, ns):
                tl.tm_cg_solve(o, x, e, n, prm)
        res[f"uneven_{name}_sequential_ms"] = timed(lambda: seq(eager))
        res[f"uneven_{name}_sequential_graph_ms"] = timed(lambda: seq(graph))
        res[f"uneven_{name}_group_ms"] = timed(lambda: tl.tm_cg_solve_group(ops, xs, etas, ns, eager))
        res[f"uneven_{name}_group_graph_ms"] = timed(lambda: tl.tm_cg_solve_group(ops, xs, etas, ns, graph))
        if name == "lp":
            # the two small lattices alone (launch-bound truncated solves)
            for j in (0, 1):
                Lr = ragged[j][0]
                tag = "x".join(str(v) for v in Lr[:1]) + "^4"
                res[f"small_lp_{tag}_eager_ms"] = timed(lambda: tl.tm_cg_solve(ops[j], xs[j], etas[j], ns[j], eager))
                res[f"small_lp_{tag}_graph_ms"] = timed(lambda: tl.tm_cg_solve(ops[j], xs[j], etas[j], ns[j], graph))
            res["small_lp_group_eager_ms"] = timed(lambda: tl.tm_cg_solve_group(ops[:2], xs[:2], etas[:2], ns[:2],
                                                                                eager))
            res["small_lp_group_graph_ms"] = timed(lambda: tl.tm_cg_solve_group(ops[:2], xs[:2], etas[:2], ns[:2],
                                                                                graph))
    for o in ops:
        o.close()
    print(json.dumps({"mode": "solvers", "steps": args.steps, "warmup": args.warmup, "results": res}),
          flush=True)


# ----------------------------------------------------------------- oracle
def _oracle_sample(c, Ls, seed):
    """One unit of the oracle's work on the sample lattice Ls: one M^dag M
    application (one CG iteration's operator work) and one source's local and
    one-derivative contractions in both one-end estimators.  Returns the two
    wall times (seconds)."""
    from oracle import loops as oloops
    from oracle.operator import apply_DW, apply_M
    from paper_1401_6749_gb300 import synth
    U = synth.gauge_field(Ls, c["gauge_seed"])
    psi = synth.random_spinor(Ls, 1, seed)[0]
    t0 = time.perf_counter()
    y = apply_M(U, apply_M(U, psi, c["kappa"], c["mu"]), c["kappa"], c["mu"], dagger=True)
    t_iter = time.perf_counter() - t0
    t0 = time.perf_counter()
    r = apply_DW(U, psi, c["kappa"])
    r[..., 2:, :] *= -1
    for left, right, mode in ((psi, psi, "vv"), (psi, r, "gen")):
        oloops.local_loops(left, right, mode)
        oloops.oneD_loops(U, left, right, mode)
    t_con = time.perf_counter() - t0
    del y
    return t_iter, t_con


def _oracle_worker(c, Ls, seed, barrier, queue):
    """A process of the all-core run: its inputs built, it waits for the
    others, then times one unit of the oracle's work."""
    _oracle_sample(c, (2, 2, 2, 2), seed)  # imports and first-touch work outside the timing
    barrier.wait()
    queue.put(_oracle_sample(c, Ls, seed))


def _oracle_all_cores(c, Ls, procs):
    """procs single-threaded processes (spawned, one per host core) each run
    one unit at the same time; returns the median per-process times."""
    import multiprocessing as mp
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        barrier, queue = ctx.Barrier(procs), ctx.Queue()
        ps = [ctx.Process(target=_oracle_worker, args=(c, Ls, 5 + i, barrier, queue)) for i in range(procs)]
        for p in ps:
            p.start()
        res = [queue.get() for _ in ps]
        for p in ps:
            p.join()
    finally:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return statistics.median(r[0] for r in res), statistics.median(r[1] for r in res)


def cpu_baseline(c, it_lp, it_hp, sample_L=(16, 16, 16, 32), all_cores=True):
    """Time the FP64 oracle, as it stands, on a bounded sample (_oracle_sample
    on a 16^3 x 32 lattice with the workload's kappa and mu), on one core and
    on all host cores (one single-threaded process per core, each running the
    same unit at the same time: the machine's throughput is procs units per
    per-process time).  The per-site cost is scaled to the workload's volume
    and combined with the iteration counts of the unpreconditioned CG (the
    oracle's algorithm; counted on this GPU for the workload, since the oracle
    cannot run it in bounded time) for the LP and HP solves to give seconds
    per source."""
    import numpy as np
    Ls = sample_L
    scale = float(np.prod(c["L"])) / float(np.prod(Ls))
    n_src = c["n_hp"] + c["n_lp"]
    iters = sum(it_lp) + sum(it_hp)

    def per_source(t_iter, t_con, procs):
        return scale * (t_iter * iters + t_con * (n_src + c["n_hp"])) / n_src / procs

    t1 = _oracle_sample(c, Ls, 5)
    one = per_source(t1[0], t1[1], 1)
    procs = os.cpu_count() or 1
    out = {"value": round(one, 3), "unit": "s/source", "cores": 1, "kind": "oracle"}
    if all_cores and procs > 1:
        tp = _oracle_all_cores(c, Ls, procs)
        out.update(value=round(per_source(tp[0], tp[1], procs), 3), cores=procs,
                   single_core={"value": round(one, 3), "unit": "s/source", "cores": 1})
    else:
        tp = t1
    out["sample"] = ("numpy FP64 oracle on %dx%dx%dx%d: one M^dag M application %.2f s, local+oneD "
                     "contractions (vv, gen) of one source %.2f s per process (1 core: %.2f s, %.2f s); "
                     "scaled by volume (x%g) and by the unpreconditioned CG iterations of the step "
                     "(%d LP + %d HP)" % (Ls + (tp[0], tp[1], t1[0], t1[1], scale, sum(it_lp), sum(it_hp))))
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    c = CONFIGS[args.config]
    # CG iteration counts per source (--ref-lp-iters / --ref-hp-iters, set to
    # those the GPU path reports for the workload) stand in for the oracle's own
    # CG, which takes the same number of iterations in exact arithmetic
    it_lp = [args.ref_lp_iters] * (c["n_hp"] + c["n_lp"])
    it_hp = [args.ref_hp_iters] * c["n_hp"]
    vals, walls = [], []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(c, it_lp, it_hp, sample_L=(8, 8, 8, 16))
        if k >= args.warmup:
            vals.append(cb["value"])
            walls.append(time.perf_counter() - t0)
    v = statistics.median(vals)
    cb["value"] = v
    n_src = c["n_hp"] + c["n_lp"]
    # a step of this arm is one bounded sample: ms_per_step is its wall time;
    # workload_ms_per_step is the oracle's time for one whole step of the
    # workload (all sources), extrapolated from the sample
    line = {"metric": METRIC, "value": v, "unit": "s/source", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(statistics.median(walls) * 1e3, 1),
            "workload_ms_per_step": round(v * n_src * 1e3, 1),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_name(c)}, "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "s/source", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", choices=sorted(CONFIGS), default="tsm32")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-baseline", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    # unpreconditioned CG iterations per source of the 32^3 x 64 workload (the
    # oracle's CG), as measured by the GPU path: LP to 1e-2, HP to 1e-9
    ap.add_argument("--ref-lp-iters", type=float, default=16)
    ap.add_argument("--ref-hp-iters", type=float, default=105)
    ap.add_argument("--schur", type=int, default=None, help="override even/odd preconditioning")
    ap.add_argument("--delta", type=float, default=None, help="override the reliable-update delta")
    ap.add_argument("--recon", type=int, default=None, choices=[0, 12, 18],
                    help="reals per link in the narrow copies; 0 = per precision")
    ap.add_argument("--overlap", type=int, default=None, help="override HP/LP stream overlap")
    ap.add_argument("--hp-ru", default=None, choices=["f64", "ff"],
                    help="override the arithmetic of the HP solves' true residuals")
    ap.add_argument("--lp-prec", default=None, choices=["f16", "bf16", "f32"])
    ap.add_argument("--hp-inner", default=None, choices=["f16", "bf16", "f32"])
    ap.add_argument("--hp-loops", default=None, choices=["f64", "ff"],
                    help="precision of the HP loops (D_W s and contractions)")
    ap.add_argument("--dslash", action="store_true", help="time tm_dslash alone")
    ap.add_argument("--next", action="store_true", help="time HPE, time dilution, momentum projection")
    ap.add_argument("--solvers", action="store_true", help="time graph-replayed and grouped solves")
    ap.add_argument("--contract", action="store_true", help="time the loop contractions alone")
    ap.add_argument("--lattice", default="32,32,32,64")
    ap.add_argument("--nrhs", type=int, default=16)
    ap.add_argument("--prec", default="f16", choices=["f64", "f32", "f16", "bf16", "ff"])
    ap.add_argument("--layout", default="std", choices=["std", "il"],
                    help="--dslash / --contract: standard layout (CUDA-core kernels) or system-interleaved (tensor cores)")
    args = ap.parse_args()
    c = CONFIGS[args.config]
    if args.schur is not None:
        c["schur"] = bool(args.schur)
    if args.delta is not None:
        c["delta"] = args.delta
    if args.overlap is not None:
        c["overlap"] = bool(args.overlap)
    if args.hp_ru is not None:
        c["hp_ru"] = args.hp_ru
    if args.recon is not None:
        c["recon"] = args.recon
    else:
        args.recon = c["recon"]
    if args.lp_prec is not None:
        c["lp_prec"] = args.lp_prec
    if args.hp_inner is not None:
        c["hp_inner"] = args.hp_inner
    if args.hp_loops is not None:
        c["hp_loops"] = args.hp_loops
    if args.dslash:
        run_dslash(args)
    elif args.next:
        run_next(args)
    elif args.solvers:
        run_solvers(args)
    elif args.contract:
        run_contract(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
