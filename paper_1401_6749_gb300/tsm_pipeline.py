"""The Truncated Solver Method loop pipeline (Sec. 2.1, Eq. 4) over the C ABI.

Orchestration only: every arithmetic step is a libtmloops kernel.

For sources r = first .. first + N_HP + N_LP - 1 (Z4, Sec. 2):
  * low-precision (LP) solves of all N_HP + N_LP sources, PLAIN CG in F16/BF16
    truncated at |r|/|b| = tol_lp, in batches of `batch` right-hand sides
    (even/odd preconditioned unless schur=False);
  * high-precision (HP) solves of the first N_HP sources, MIXED CG (FP64
    reliable updates) to tol_hp;
  * for every solution s: local and one-derivative loops with the one-end
    trick (L = R = s, P = g5, Eq. 5) and its generalisation (L = s,
    R = g5 D_W s, P = g5, Eq. 6); for the HP solutions D_W s and the
    contractions run in hp_loop_prec: F64, or FF (float-float, about 48 bits
    on the FP32 pipes, after one conversion of the FP64 solution), whose
    loops agree with the FP64 ones to ~1e-13 relative;
  * TSM combination with prefactor -2 i nu (one-end) and 2 (generalised).
The LP solve of a source is the same function of the source in every batch
(per-system arithmetic, fixed-order reductions), so the correction term of
Eq. 4 is unbiased.
"""
import threading

import torch

from . import tmloops as tl

KINDS = ("local_vv", "local_gen", "oneD_vv", "oneD_gen")


class TsmPipeline:
    def __init__(self, op, n_hp, n_lp, batch=16, lp_prec=tl.F16, hp_inner=tl.F32, tol_lp=1e-2,
                 tol_hp=1e-9, seed=20140126, first_src=0, max_iter=20000, check_every=4,
                 delta=0.1, kinds=KINDS, schur=True, overlap=False, hp_loop_prec=tl.F64, timing=False,
                 lp_layout=None, lp_graph=None, hp_ru_prec=None, hp_first=False):
        """lp_layout: "il" draws the LP sources straight into the
        system-interleaved layout (z4_noise_il), solves there (tm_cg_solve_il),
        applies D_W there (tm_dslash_il) and contracts
        there (loop_contract_*_il, gamma_5 of the generalised estimator as
        right_g5); "std" uses the standard layout throughout.  Default: "il"
        for FP16/BF16 with 18-real 16-bit links (recon 18 or 0), else "std".
        hp_first: without overlap, run the HP solves and loops before the LP
        batches instead of after them (the sources are independent: every
        per-source result is the same in either order).
        hp_ru_prec: arithmetic of the HP solves' true residuals (reliable
        updates), F64 (default) or FF.  FF is exact to about 2^-48 cond(M^dag M)
        relative to |b|: only for solves well enough conditioned that this
        stays far below tol_hp.
        lp_graph: replay the truncated LP solves' iterations as CUDA graphs
        (bit-identical; the operator keeps the graph for the next batch).
        Default: on where launches weigh (half volume <= 2^17 sites), off on
        larger lattices, whose kernels run for a millisecond or more.
        overlap: run the high-precision solves and contractions on a second
        stream from a host thread, concurrently with the low-precision batches
        (FP64 work uses other units than the FP32 arithmetic of the LP solves);
        needs its own operator handle (a clone sharing the links).
        timing: record CUDA events around the phases of every batch (solve,
        local loops with the D_W of the generalised estimator, one-derivative
        loops), read by phase_ms() after a run."""
        self.op = op
        self.overlap = bool(overlap)
        self.op_hp = op.clone() if self.overlap else op
        self.hp_stream = torch.cuda.Stream() if self.overlap else None
        self.L = op.L
        self.T = op.L[3]
        self.n_hp, self.n_lp = int(n_hp), int(n_lp)
        self.batch = int(batch)
        self.lp_prec, self.hp_inner = lp_prec, hp_inner
        self.tol_lp, self.tol_hp = tol_lp, tol_hp
        self.seed, self.first = int(seed), int(first_src)
        self.max_iter, self.check_every, self.delta = max_iter, check_every, delta
        self.schur = bool(schur)
        self.hp_first = bool(hp_first)
        if hp_loop_prec not in (tl.F64, tl.FF):
            raise ValueError("hp_loop_prec must be F64 or FF")
        self.hp_loop_prec = hp_loop_prec
        self.hp_ru_prec = tl.F64 if hp_ru_prec is None else hp_ru_prec
        if self.hp_ru_prec not in (tl.F64, tl.FF):
            raise ValueError("hp_ru_prec must be F64 or FF")
        self.kinds = tuple(kinds)
        il_ok = lp_prec in (tl.F16, tl.BF16) and op.recon in (0, 18)
        if lp_layout is None:
            lp_layout = "il" if il_ok else "std"
        if lp_layout not in ("il", "std") or (lp_layout == "il" and not il_ok):
            raise ValueError("lp_layout 'il' needs F16/BF16 and 18-real 16-bit links; 'std' always works")
        self.lp_il = lp_layout == "il"
        vh = op.L[0] * op.L[1] * op.L[2] * op.L[3] // 2
        self.lp_graph = (vh <= 1 << 17) if lp_graph is None else bool(lp_graph)
        self.nu = 2.0 * op.kappa * op.mu
        n_all = self.n_hp + self.n_lp
        self.len = {"local": 16 * self.T, "oneD": 64 * self.T}
        dev = "cuda"
        # per-source loop arrays (complex as re/im doubles)
        self.lp_loops = {k: torch.empty((n_all, self.len[k.split("_")[0]] * 2), dtype=torch.float64,
                                        device=dev) for k in self.kinds}
        self.hp_loops = {k: torch.empty((max(self.n_hp, 1), self.len[k.split("_")[0]] * 2),
                                        dtype=torch.float64, device=dev) for k in self.kinds}
        b = min(self.batch, n_all)
        if self.lp_il:
            self._lp = [tl.empty_field_il(self.L, b) for _ in range(3)]  # eta, x, D_W x (interleaved)
        else:
            self._lp = [tl.empty_field(self.L, lp_prec, b) for _ in range(3)]  # eta, x, g5 D_W x
        nh = max(min(self.batch, self.n_hp), 1)
        # eta, x, g5 D_W x (the last in hp_loop_prec, same byte size), and the copies of
        # eta and x in hp_loop_prec when that is not F64
        nf = 3 if hp_loop_prec == tl.F64 else 5
        self._hp = [tl.empty_field(self.L, tl.F64, nh) for _ in range(nf)] if self.n_hp else None
        self.stats_lp, self.stats_hp = [], []
        self.timing = bool(timing)
        self._events = []  # (set "lp"/"hp", [e_start, e_solved, e_local, e_oned])

    def _event(self, stream):
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream if stream is not None else torch.cuda.current_stream())
        return e

    def phase_ms(self):
        """Device milliseconds of the last run per set and phase:
        {"lp": {"solve", "local", "oneD"}, "hp": {...}} (synchronises)."""
        torch.cuda.synchronize()
        out = {k: {"solve": 0.0, "local": 0.0, "oneD": 0.0} for k in ("lp", "hp")}
        for which, ev in self._events:
            out[which]["solve"] += ev[0].elapsed_time(ev[1])
            out[which]["local"] += ev[1].elapsed_time(ev[2])
            out[which]["oneD"] += ev[2].elapsed_time(ev[3])
        return out

    def _contract(self, op, x, g5w, prec, n, dst, row0, stream, eta=None, kinds=None):
        for k in (self.kinds if kinds is None else kinds):
            kind, mode = k.split("_")
            left, right = {"vv": (x, x), "gen": (x, g5w), "std": (eta, x)}[mode]
            out = dst[k][row0:row0 + n]
            if kind == "local":
                tl.loop_contract_local(self.L, left, right, prec, n, tl.LOOP_MODE[mode], out, stream)
            else:
                tl.loop_contract_oneD(op, left, right, prec, n, tl.LOOP_MODE[mode], out, stream)

    def _contract_il(self, op, x, dw, eta, prec, n, dst, row0, stream, kinds):
        for k in kinds:
            kind, mode = k.split("_")
            left, right, g5 = {"vv": (x, x, False), "gen": (x, dw, True), "std": (eta, x, False)}[mode]
            out = dst[k][row0:row0 + n]
            if kind == "local":
                tl.loop_contract_local_il(self.L, left, right, prec, n, tl.LOOP_MODE[mode], out, right_g5=g5,
                                          stream=stream)
            else:
                tl.loop_contract_oneD_il(op, left, right, prec, n, tl.LOOP_MODE[mode], out, right_g5=g5,
                                         stream=stream)

    def _solve_and_contract_il(self, op, fields, prec, first, n, params, dst, row0, stream=None):
        """An LP batch on the interleaved layout: solve, D_W, contractions."""
        eta_il, x, dw = fields
        ev = [self._event(stream)] if self.timing else None
        tl.z4_noise_il(self.L, eta_il, prec, self.seed, first, n, stream)
        st, stats = tl.tm_cg_solve_il(op, x, eta_il, n, params, stream, raise_on_noconv=False)
        if ev:
            ev.append(self._event(stream))
        if any("gen" in k for k in self.kinds):
            tl.tm_dslash_il(op, dw, x, n, mu_zero=True, prec=prec, stream=stream)   # D_W s
        local = tuple(k for k in self.kinds if k.startswith("local"))
        oned = tuple(k for k in self.kinds if k.startswith("oneD"))
        self._contract_il(op, x, dw, eta_il, prec, n, dst, row0, stream, local)
        if ev:
            ev.append(self._event(stream))
        self._contract_il(op, x, dw, eta_il, prec, n, dst, row0, stream, oned)
        if ev:
            ev.append(self._event(stream))
            self._events.append(("lp", ev))
        return stats

    def _solve_and_contract(self, op, fields, prec, first, n, params, dst, row0, stream=None,
                            loop_prec=None, which="lp"):
        eta, x, g5w = fields[:3]
        ev = [self._event(stream)] if self.timing else None
        tl.z4_noise(self.L, eta, prec, self.seed, first, n, stream)
        st, stats = tl.tm_cg_solve(op, x, eta, n, params, stream, raise_on_noconv=False)
        if loop_prec is not None and loop_prec != prec:
            # one conversion of the solution (and source) to the loop precision
            eta_l, x_l = fields[3], fields[4]
            tl.tm_spinor_convert(self.L, x_l, loop_prec, x, prec, n, stream)
            if any(k.endswith("std") for k in self.kinds):
                tl.tm_spinor_convert(self.L, eta_l, loop_prec, eta, prec, n, stream)
            eta, x, prec = eta_l, x_l, loop_prec
        if ev:
            ev.append(self._event(stream))
        if any("gen" in k for k in self.kinds):
            tl.tm_dslash_g5(op, g5w, x, n, mu_zero=True, prec=prec, stream=stream)   # g5 D_W s
        local = tuple(k for k in self.kinds if k.startswith("local"))
        oned = tuple(k for k in self.kinds if k.startswith("oneD"))
        self._contract(op, x, g5w, prec, n, dst, row0, stream, eta, local)
        if ev:
            ev.append(self._event(stream))
        self._contract(op, x, g5w, prec, n, dst, row0, stream, eta, oned)
        if ev:
            ev.append(self._event(stream))
            self._events.append((which, ev))
        return stats

    def _run_hp(self, stream):
        hp_params = tl.cg_params(self.tol_hp, self.max_iter, tl.CG_MIXED, inner_prec=self.hp_inner,
                                 delta=self.delta, check_every=self.check_every, schur=self.schur,
                                 ru_prec=self.hp_ru_prec)
        stats = []
        for b0 in range(0, self.n_hp, self.batch):
            n = min(self.batch, self.n_hp - b0)
            stats += self._solve_and_contract(self.op_hp, self._hp, tl.F64, self.first + b0, n,
                                              hp_params, self.hp_loops, b0, stream,
                                              loop_prec=self.hp_loop_prec, which="hp")
        self.stats_hp = stats

    def run(self, dist=None):
        """One full TSM estimate; returns per-kind (mean, err) device tensors.

        With a torch.distributed module whose world size exceeds one, every rank
        runs its own sources (first_src set per rank) and the estimate combines
        the sources of all ranks (one all-gather of the per-source loops)."""
        self.run_sources()
        if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
            return self.combine_global(dist)
        return self.combine()

    def run_sources(self):
        """The solves and contractions of every source (per-source loops in
        lp_loops / hp_loops), without the combination."""
        n_all = self.n_hp + self.n_lp
        self.stats_lp, self.stats_hp = [], []
        self._events = []
        main = torch.cuda.current_stream()
        worker = None
        if self.n_hp and self.overlap:
            # the HP stream starts after everything queued before this step
            self.hp_stream.wait_stream(main)
            worker = threading.Thread(target=self._run_hp, args=(self.hp_stream,))
            worker.start()
        # the truncated solves stop after a handful of iterations: poll often so
        # that no masked-out iterations are launched past convergence
        lp_params = tl.cg_params(self.tol_lp, self.max_iter, tl.CG_PLAIN, prec=self.lp_prec,
                                 check_every=min(2, self.check_every), schur=self.schur, graph=self.lp_graph)
        if self.n_hp and worker is None and self.hp_first:
            self._run_hp(main)
        for b0 in range(0, n_all, self.batch):
            n = min(self.batch, n_all - b0)
            if self.lp_il:
                self.stats_lp += self._solve_and_contract_il(self.op, self._lp, self.lp_prec, self.first + b0, n,
                                                             lp_params, self.lp_loops, b0, main)
            else:
                self.stats_lp += self._solve_and_contract(self.op, self._lp, self.lp_prec, self.first + b0, n,
                                                          lp_params, self.lp_loops, b0, main)
        if worker is not None:
            worker.join()
            main.wait_stream(self.hp_stream)
        elif self.n_hp and not self.hp_first:
            self._run_hp(main)

    def _combine_sets(self, k, hp, lphp, lp, n_hp, n_lp):
        length = self.len[k.split("_")[0]]
        scale = -2j * self.nu if k.endswith("vv") else 2.0
        mean = torch.empty(2 * length, dtype=torch.float64, device="cuda")
        err = torch.empty(2 * length, dtype=torch.float64, device="cuda")
        if n_hp:
            tl.tsm_combine(hp, lphp, n_hp, lp, n_lp, length, scale, mean, err)
        else:
            tl.tsm_combine(None, None, 0, lp, n_lp, length, scale, mean, err)
        return mean, err

    def combine(self):
        """TSM estimate (Eq. 4) from this process's sources."""
        res = {}
        for k in self.kinds:
            lp = self.lp_loops[k]
            res[k] = self._combine_sets(k, self.hp_loops[k][:self.n_hp], lp[:self.n_hp],
                                        lp[self.n_hp:], self.n_hp, self.n_lp)
        return res

    def combine_global(self, dist):
        """TSM estimate over the sources of all ranks (one all-gather per kind)."""
        from .distributed import gather_tsm_sets
        world = dist.get_world_size()
        res = {}
        for k in self.kinds:
            hp_all, lphp, lp = gather_tsm_sets(dist, self.hp_loops[k][:self.n_hp], self.lp_loops[k],
                                               self.n_hp)
            res[k] = self._combine_sets(k, hp_all, lphp, lp, world * self.n_hp, world * self.n_lp)
        return res
