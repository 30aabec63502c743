"""Benchmark of the Wilson-clover hot path on GB300.

Workload: the 48x24^3 lattice of Sec. 3 (kappa = 0.13625, c_sw = 1.9,
synthetic SU(3) links with plaquette 0.55, antiperiodic time), 12 Gaussian
right-hand sides batched in one multi-RHS stencil.  One step = one application
of the even-odd Schur complement Dhat (Eq. 2) in FP32 to the 12-field batch,
on fields resident in HBM in the library's native layout.

value    : Dhat GFLOP/s (3672 flop per even site per field)
e2e      : the same through the public C ABI (lqcd_apply_Dhat on canonical
           fields) with the step's sources copied host->device from pinned
           memory and the result read back inside the timed region
roofline : algorithmic HBM bytes of one Dhat application / its CUDA-event time
cpu_baseline: the FP64 CPU oracle's Dhat on the same lattice (1 field)

`--impl reference` times the CPU oracle alone (the comparison arm).
Several GPUs (torchrun): independent replicas, one lattice batch per rank.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLOP_PER_SITE = 3672
DIMS = (48, 24, 24, 24)
KAPPA, CSW = 0.13625, 1.9
WORKLOAD = "48x24^3 Wilson-clover Dhat_ee, kappa=0.13625, c_sw=1.9, 12 RHS"


def dhat_bytes_per_site(prec: str, nrhs: int) -> int:
    """Algorithmic HBM bytes of one Dhat application per even site, all fields.
    Links: each of the two half-hops reads every link once (8 per site);
    clover: A_ee and A_oo^-1 (2 x 72 reals); per field: psi_e read by both
    kernels, chi_o written and read, out written (5 x 24 reals)."""
    if prec == "f16s":   # FP16 links (2 rows) and clover; a field site is 48 B of halves + a 4 B scale
        return 2 * (2 * 8 * 12 + 144) + 5 * 52 * nrhs
    word = 8 if prec == "f64" else 4
    link_words = 2 * 8 * (18 if prec == "f64" else 12)
    return word * (link_words + 144 + 120 * nrhs)


# ncu DRAM bytes (read + write) of one Dhat application per even site, FP32 with
# 12 fields, from the full-size 48x24^3 capture summarised in profiles/ (mean of
# two applications; valid for the FMA-chain stencil kernels it was taken of)
TRAFFIC_F32_12_PER_SITE = 2558.6e6 / 331776
TRAFFIC_NOTE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the tuned DHAT1 + DHAT2 stencil kernels "
                "at 48x24^3 x 12 fields (2558.6 MB per application, 1.086 x algorithmic)")


def traffic_of(prec, nrhs, Vh):
    if prec == "f32" and nrhs == 12:
        return int(TRAFFIC_F32_12_PER_SITE * Vh)
    return None


def max_over_ranks(ms: float, dist=None, device="cuda") -> float:
    """The slowest rank's duration of the timed region (every rank returns it);
    one process per GPU, replicas only: this is the only collective."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step: float, steps: int, world: int, max_ms: float) -> float:
    """Units processed by all ranks per second of the slowest rank's timed region."""
    return units_per_rank_step * steps * world / (max_ms * 1e-3)


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d["hbm_gbs"], "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.p = None
        self.out = []

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            txt, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            txt, _ = self.p.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in txt.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(steps: int = 2):
    """The FP64 oracle's Dhat on the same 48x24^3 lattice (one field): a bounded
    sample of the workload, scaled to GFLOP/s."""
    import oracle as orc
    from paper_1011_0911_gb300 import synth
    U = synth.su3_links(DIMS, 0)
    o = orc.Oracle(DIMS, U, KAPPA, CSW)
    pe = synth.gaussian_spinor(o.Vh, 1)
    o.Dhat(pe)
    t0 = time.perf_counter()
    for _ in range(steps):
        o.Dhat(pe)
    dt = (time.perf_counter() - t0) / steps
    return {"value": round(FLOP_PER_SITE * o.Vh / dt / 1e9, 4), "unit": "GFLOP/s", "cores": orc.num_threads(),
            "kind": "oracle",
            "sample": f"{steps} FP64 Dhat applications on one 48x24^3 field (one-field sample of the 12-field step)",
            "seconds_per_application": round(dt, 4)}


KAPPA_OF = {(8, 8, 8, 8): 0.1355, (32, 16, 16, 16): 0.1357, (48, 24, 24, 24): 0.13625, (64, 32, 32, 32): 0.1363}


def solve_once(ctx, lqcd, eta, solver, inner, Ns=20, ninv=8, ctol=1e-2, seed=100, cnmx=4096, cnkv=16, cprec=None,
               nkv=16, sap_prec=None, krylov=None, ncy=4, nmr=5, bncy=4, bnmr=4, bprec=None, ceo=False):
    """Time-to-solution of Dhat psi = eta (all fields of eta) to 1e-10 with the
    given solver; the subspace build is timed separately and included in total."""
    import torch
    from paper_1011_0911_gb300 import synth
    prec = lqcd.F32 if inner == "f32" else lqcd.F64
    res = {"solver": solver, "inner": inner, "nrhs": int(eta.shape[0])}
    torch.cuda.synchronize()
    build_s = 0.0
    if solver == "dfl":
        v0 = torch.from_numpy(synth.gaussian_spinor(Ns * ctx.V, seed, synth.STREAM_SUBSPACE)
                              .reshape(Ns, ctx.V, 4, 3)).cuda()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        l0 = ctx.kernel_launches
        cp = prec if cprec is None else (lqcd.F32 if cprec == "f32" else lqcd.F64)
        ctx.dfl_build(v0, bs=(4, 4, 4, 4), ninv=ninv, ncy=bncy, nmr=bnmr, prec=prec, coarse_tol=ctol,
                      build_sap_prec=bprec, coarse_eo=ceo,
                      coarse_nkv=cnkv, coarse_nmx=cnmx, coarse_prec=cp)
        torch.cuda.synchronize()
        build_s = time.perf_counter() - t0
        res.update({"Ns": Ns, "ninv": ninv, "build_sap": [bncy, bnmr], "coarse_tol": ctol, "coarse_nmx": cnmx,
                    "coarse_nkv": cnkv, "coarse_eo": bool(ceo),
                    "coarse_prec": "f32" if cp == lqcd.F32 else "f64", "build_s": round(build_s, 4),
                    "build_launches": ctx.kernel_launches - l0})
    sid = {"cgnr": lqcd.SOLVER_CGNR, "sap": lqcd.SOLVER_SAP_GCR, "dfl": lqcd.SOLVER_DFL_SAP_GCR}[solver]
    t0 = time.perf_counter()
    l0 = ctx.kernel_launches
    sp = prec if sap_prec is None else sap_prec
    kr = lqcd.F32 if krylov == "f32" else lqcd.F64
    psi, info, st = ctx.solve_dhat(eta, solver=sid, tol=1e-10, nmx=20000 if solver == "cgnr" else 4096,
                                   nkv=nkv, sap_prec=sp, inner=prec, check=False, krylov=kr, ncy=ncy, nmr=nmr)
    torch.cuda.synchronize()
    solve_s = time.perf_counter() - t0
    res.update({"krylov": "f32" if kr == lqcd.F32 else "f64", "solve_launches": ctx.kernel_launches - l0,
                "status": st, "solve_s": round(solve_s, 4), "total_s": round(solve_s + build_s, 4),
                "iters": [i["iters"] for i in info],
                "max_relres_dhat": max(i["relres_dhat"] for i in info)})
    if solver == "dfl":
        res["coarse_solves"], res["coarse_iters"] = ctx.dfl_stats()
    return res, psi


# solver parameters of every deflated form of the time-to-solution table (the
# forms differ only in precision and batching): Ns = 20 subspace fields built by
# 6 inverse iterations of SAP with 6 cycles x 4 MinRes steps, SAP smoother with
# 1 cycle x 4 MinRes steps, little-Dirac GCR of 64 steps with Krylov length 32
# (32 steps in the even-odd form used with the FP32 little operator), chosen by
# timing whole 12-source solves at 48x24^3 (bench.py --mode solve with
# --ninv/--bncy/--bnmr/--ncy/--nmr/--cnmx/--cnkv/--ceo)
DFL_NINV, DFL_BUILD_SAP, DFL_SAP, DFL_CNMX, DFL_CNKV = 6, (6, 4), (1, 4), 64, 32
DFL_CEO, DFL_CNMX_EO = True, 32


def time_to_solve(ctx, lqcd, eta, net=None):
    """Time-to-solution of Dhat psi = eta for the 12 sources to a true relative
    residual <= 1e-10 (checked in FP64), subspace builds included:
      plain_f64 : deflated SAP-GCR, FP64 everywhere, one source at a time
      dfl_mixed : deflated SAP-GCR with the workload's stated precisions: FP32
                  SAP, subspace and stencil, FP64 outer GCR (Krylov vectors and
                  Gram-Schmidt) and FP64 little-Dirac solve, the 12 sources in
                  one batched solve
      chosen    : the fastest measured form: FP16 (per-site scale) SAP, FP32
                  subspace, stencil, little-Dirac solve and GCR Krylov vectors
                  (FP64 residual, solution and restarts), 12 sources batched
      learned   : the chosen form's subspace and precisions with the trained
                  network as the smoother (deflated SAP where its step fails);
                  training at 32x16^3 reported apart
      sap_f32, sap_f16s : SAP-GCR without deflation, FP32 / FP16 SAP, FP64 GCR
    Every form is first run for two steps (and its subspace built once) so
    that launch-shape tuning and workspace growth stay out of the timings."""
    import torch
    from paper_1011_0911_gb300 import synth
    out = {}
    one = eta[:1].contiguous()
    for spr, inner in ((lqcd.F32, lqcd.F32), (lqcd.F16S, lqcd.F32), (lqcd.F64, lqcd.F64)):
        ctx.solve_dhat(eta, solver=lqcd.SOLVER_SAP_GCR, tol=1e-10, nmx=2, sap_prec=spr, inner=inner, check=False)
    v0 = torch.from_numpy(synth.gaussian_spinor(20 * ctx.V, 100, synth.STREAM_SUBSPACE).reshape(20, ctx.V, 4, 3)).cuda()
    sncy, snmr = DFL_SAP
    for prec in (lqcd.F64, lqcd.F32):
        ctx.dfl_build(v0, bs=(4, 4, 4, 4), ninv=1, ncy=DFL_BUILD_SAP[0], nmr=DFL_BUILD_SAP[1], prec=prec,
                      coarse_tol=1e-2, coarse_nmx=DFL_CNMX, coarse_nkv=DFL_CNKV, coarse_prec=prec, coarse_eo=DFL_CEO)
        e = one if prec == lqcd.F64 else eta
        ctx.solve_dhat(e, solver=lqcd.SOLVER_DFL_SAP_GCR, tol=1e-10, nmx=2, sap_prec=prec, inner=prec, check=False,
                       ncy=sncy, nmr=snmr)
        if prec == lqcd.F32:
            ctx.solve_dhat(eta, solver=lqcd.SOLVER_DFL_SAP_GCR, tol=1e-10, nmx=2, sap_prec=lqcd.F16S, inner=prec,
                           check=False, krylov=lqcd.F32, ncy=sncy, nmr=snmr)
        if prec == lqcd.F32 and net is not None:
            ctx.net_set(NET_CHANS, net["W"], act=lqcd.BF16)
            ctx.solve_dhat(eta, solver=lqcd.SOLVER_DFL_NET_GCR, tol=1e-10, nmx=2, sap_prec=prec, inner=prec,
                           check=False, krylov=lqcd.F32, ncy=sncy, nmr=snmr)
    del v0
    torch.cuda.synchronize()
    r, _ = solve_once(ctx, lqcd, eta, "sap", "f32")
    out["sap_f32"] = {"form": "SAP-GCR, FP32 SAP/stencil, FP64 GCR, 12 RHS batched", "seconds": r["total_s"],
                      "iters": max(r["iters"]), "max_relres_dhat": r["max_relres_dhat"], "status": r["status"]}
    t0 = time.perf_counter()
    _, info, st = ctx.solve_dhat(eta, solver=lqcd.SOLVER_SAP_GCR, tol=1e-10, sap_prec=lqcd.F16S, inner=lqcd.F32,
                                 check=False)
    torch.cuda.synchronize()
    out["sap_f16s"] = {"form": "SAP-GCR, FP16 (per-site scale) SAP, FP32 stencil, FP64 GCR, 12 RHS batched",
                       "seconds": round(time.perf_counter() - t0, 4), "iters": max(i["iters"] for i in info),
                       "max_relres_dhat": max(i["relres_dhat"] for i in info), "status": st}
    # the workload's stated precisions: its own subspace build (FP64 little operator)
    dflp = dict(Ns=20, ninv=DFL_NINV, ctol=1e-2, cnmx=DFL_CNMX, cnkv=DFL_CNKV, ncy=sncy, nmr=snmr,
                bncy=DFL_BUILD_SAP[0], bnmr=DFL_BUILD_SAP[1], ceo=DFL_CEO)
    r, _ = solve_once(ctx, lqcd, eta, "dfl", "f32", cprec="f64", **dflp)
    out["dfl_mixed"] = {"form": "deflated SAP-GCR (Ns=20, 4^4 blocks), FP32 SAP/subspace/stencil, FP64 GCR "
                                "(Krylov vectors, Gram-Schmidt) and FP64 little-Dirac solve, 12 RHS batched",
                        "seconds": r["total_s"], "build_s": r["build_s"], "iters": max(r["iters"]),
                        "max_relres_dhat": r["max_relres_dhat"], "status": r["status"]}
    if net is not None:
        # the same subspace and precisions (FP64 Gram-Schmidt and little-Dirac
        # solve), the trained network as the smoother in place of SAP
        ctx.net_set(NET_CHANS, net["W"], act=lqcd.BF16)
        ctx.solve_dhat(eta, solver=lqcd.SOLVER_DFL_NET_GCR, tol=1e-10, nmx=2, sap_prec=lqcd.F32, inner=lqcd.F32,
                       check=False, ncy=sncy, nmr=snmr)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, info, st = ctx.solve_dhat(eta, solver=lqcd.SOLVER_DFL_NET_GCR, tol=1e-10, sap_prec=lqcd.F32,
                                     inner=lqcd.F32, check=False, ncy=sncy, nmr=snmr)
        torch.cuda.synchronize()
        out["learned_mixed"] = {"form": "dfl_mixed's subspace and precisions (FP64 GCR and little-Dirac solve), "
                                        "trained BF16 network as smoother, deflated FP32 SAP as fallback, "
                                        "12 RHS batched",
                                "seconds": round(time.perf_counter() - t0 + r["build_s"], 4), "build_s": r["build_s"],
                                "iters": max(i["iters"] for i in info),
                                "net_fallbacks": sum(i["net_fallbacks"] for i in info),
                                "max_relres_dhat": max(i["relres_dhat"] for i in info), "status": st,
                                "training_s": net["train_s"]}
    # one subspace build with the FP32 little operator (timed, included in both
    # forms below) and two smoothers on it
    r, _ = solve_once(ctx, lqcd, eta, "dfl", "f32", cprec="f32", sap_prec=lqcd.F16S, krylov="f32", bprec=lqcd.F16S,
                      **dict(dflp, cnmx=DFL_CNMX_EO if DFL_CEO else DFL_CNMX))
    build = r["build_s"]
    out["chosen"] = {"form": "deflated SAP-GCR (Ns=20, 4^4 blocks), FP16 (per-site scale) SAP in the solve and the "
                             "subspace build, FP32 subspace, "
                             "stencil, even-odd little-Dirac solve and GCR Krylov vectors; FP64 residual, "
                             "solution and restarts; 12 RHS batched",
                     "seconds": r["total_s"], "build_s": build, "iters": max(r["iters"]), "net_fallbacks": 0,
                     "max_relres_dhat": r["max_relres_dhat"], "status": r["status"]}
    if net is not None:
        # the same subspace, the network in place of the SAP smoother
        ctx.net_set(NET_CHANS, net["W"], act=lqcd.BF16)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, info, st = ctx.solve_dhat(eta, solver=lqcd.SOLVER_DFL_NET_GCR, tol=1e-10, sap_prec=lqcd.F32,
                                     inner=lqcd.F32, check=False, krylov=lqcd.F32, ncy=sncy, nmr=snmr)
        torch.cuda.synchronize()
        out["learned"] = {"form": "deflated GCR (Ns=20), trained BF16 network as smoother, deflated FP32 SAP as "
                                  "fallback, the chosen form's FP32 subspace / little-Dirac solve / Krylov vectors, "
                                  "12 RHS batched",
                          "seconds": round(time.perf_counter() - t0 + build, 4), "build_s": build,
                          "iters": max(i["iters"] for i in info),
                          "net_fallbacks": sum(i["net_fallbacks"] for i in info),
                          "max_relres_dhat": max(i["relres_dhat"] for i in info), "status": st,
                          "training": {"lattice": "32x16x16x16", "pairs": net["pairs"], "seconds": net["train_s"],
                                       "loss_first": net["loss_first"], "loss_last": net["loss_last"],
                                       "residual_loss_last": net.get("residual_loss_last")}}
    total, build, iters, worst, st = 0.0, 0.0, 0, 0.0, 0
    for k in range(eta.shape[0]):
        if k == 0:
            r, _ = solve_once(ctx, lqcd, eta[k:k + 1].contiguous(), "dfl", "f64", cprec="f64", **dflp)
            build = r["build_s"]
            total += r["total_s"]
        else:   # the subspace is reused for the other sources
            sid = lqcd.SOLVER_DFL_SAP_GCR
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            psi, info, s = ctx.solve_dhat(eta[k:k + 1].contiguous(), solver=sid, tol=1e-10, sap_prec=lqcd.F64,
                                          inner=lqcd.F64, check=False, ncy=sncy, nmr=snmr)
            torch.cuda.synchronize()
            total += time.perf_counter() - t0
            r = {"iters": [info[0]["iters"]], "max_relres_dhat": info[0]["relres_dhat"], "status": s}
        iters = max(iters, max(r["iters"]))
        worst = max(worst, r["max_relres_dhat"])
        st = st or r["status"]
    out["plain_f64"] = {"form": "deflated SAP-GCR (Ns=20, 4^4 blocks), FP64 throughout, one source at a time",
                        "seconds": round(total, 4), "build_s": build, "iters": iters, "max_relres_dhat": worst,
                        "status": st}
    for k in ("chosen", "sap_f32", "sap_f16s", "dfl_mixed", "learned", "learned_mixed"):
        if k in out:
            out["speedup_%s_vs_plain_f64" % k] = round(out["plain_f64"]["seconds"] / out[k]["seconds"], 2)
    if "learned_mixed" in out:
        out["gain_learned_mixed_vs_dfl_mixed"] = round(out["dfl_mixed"]["seconds"] / out["learned_mixed"]["seconds"], 3)
    if "learned" in out:
        out["gain_learned_vs_chosen"] = round(out["chosen"]["seconds"] / out["learned"]["seconds"], 3)
    out["tolerance"] = 1e-10
    return out


def run_solve(args):
    import torch
    from paper_1011_0911_gb300 import lqcd, synth
    kappa = args.kappa or KAPPA_OF.get(DIMS, 0.1355)
    ctx = lqcd.Context(DIMS)
    ctx.set_gauge(torch.from_numpy(synth.su3_links(DIMS, 0)).cuda())
    ctx.clover_invert(kappa, CSW)
    eta = torch.from_numpy(synth.gaussian_spinor(args.nrhs * ctx.Vh, 1).reshape(args.nrhs, ctx.Vh, 4, 3)).cuda()
    # the first pass tunes launch shapes and grows workspaces; the second is reported
    l0 = ctx.kernel_launches
    for p in range(2):
        if p == 1:
            first_pass_launches = ctx.kernel_launches - l0
        res, _ = solve_once(ctx, lqcd, eta, args.solver, args.prec, Ns=args.Ns, ninv=args.ninv, ctol=args.ctol,
                            cnmx=args.cnmx, cnkv=args.cnkv, cprec=args.cprec, nkv=args.nkv,
                            krylov=args.krylov, ncy=args.ncy, nmr=args.nmr, bncy=args.bncy, bnmr=args.bnmr,
                            bprec={"f16s": lqcd.F16S, "f32": lqcd.F32}.get(args.bprec), ceo=args.ceo,
                            sap_prec={"f16s": lqcd.F16S, "f32": lqcd.F32, "f64": lqcd.F64}.get(args.sap_prec))
    res["first_pass_launches"] = first_pass_launches
    res["nkv"] = args.nkv
    res["ncy"], res["nmr"] = args.ncy, args.nmr
    res["sap_prec"] = args.sap_prec or args.prec
    res.update({"mode": "solve", "lattice": args.lattice, "kappa": kappa})
    print(json.dumps(res))


BATCH_SIZES = [(8, 8, 8, 8), (16, 16, 16, 16), (24, 12, 12, 12), (32, 16, 16, 16)]


def run_batch(args):
    """Uneven batch of lattices drawn with a seeded host generator from four
    sizes, kappa uniform in [0.1350, 0.1360], c_sw = 1.9, one Gaussian source
    each; FP16 (per-site scale) SAP, FP32 stencil, FP64 GCR, tolerance 1e-10
    per lattice.  The batched solver (one launch per phase over all lattices,
    cycles replayed from a CUDA graph) is timed against solving the same
    lattices one after the other with the single-lattice solver."""
    import numpy as np
    import torch
    from paper_1011_0911_gb300 import lqcd, synth
    rng = np.random.default_rng(0)
    picks = rng.integers(0, len(BATCH_SIZES), args.nlat)
    kappas = rng.uniform(0.1350, 0.1360, args.nlat)
    lats = [(BATCH_SIZES[int(i)], float(k)) for i, k in zip(picks, kappas)]
    ctxs, etas = [], []
    for i, (d, k) in enumerate(lats):
        c = lqcd.Context(d)
        c.set_gauge(torch.from_numpy(synth.su3_links(d, i)).cuda())
        c.clover_invert(k, CSW)
        ctxs.append(c)
        etas.append(torch.from_numpy(synth.gaussian_spinor(c.Vh, 100 + i)).cuda())
    B = lqcd.Batch(ctxs, nkv=16, nmx=4096, tol=1e-10, sap_prec=lqcd.F16S, use_graph=not args.no_graph)
    B.solve_dhat(etas)   # warm-up: launch shapes tuned, graph captured
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    psis, info, st = B.solve_dhat(etas)
    torch.cuda.synchronize()
    batched_s = time.perf_counter() - t0
    stats = B.stats()

    def sequential():
        out = []
        for c, e in zip(ctxs, etas):
            _, inf, s1 = c.solve_dhat(e, solver=lqcd.SOLVER_SAP_GCR, tol=1e-10, nkv=16, sap_prec=lqcd.F16S,
                                      inner=lqcd.F32, check=False)
            out.append((inf[0], s1))
        return out
    sequential()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seq = sequential()
    torch.cuda.synchronize()
    seq_s = time.perf_counter() - t0
    res = {"mode": "batch", "lattices": [{"dims": "x".join(map(str, d)), "kappa": round(k, 6)} for d, k in lats],
           "form": "SAP-GCR, F16S SAP (4^4 blocks, ncy=4, nmr=5), FP32 stencil, FP64 GCR, nkv=16",
           "batched_s": round(batched_s, 4), "sequential_s": round(seq_s, 4),
           "speedup_batched_vs_sequential": round(seq_s / batched_s, 2),
           "batched_status": st, "batched_iters": [i["iters"] for i in info],
           "batched_max_relres_dhat": max(i["relres_dhat"] for i in info),
           "sequential_iters": [i["iters"] for i, _ in seq],
           "sequential_max_relres_dhat": max(i["relres_dhat"] for i, _ in seq),
           "sequential_status": max(s1 for _, s1 in seq), **stats,
           "total_sites": int(sum(c.V for c in ctxs))}
    print(json.dumps(res))


NET_CHANS = (1, 2, 2, 1)


def train_net(lqcd, synth, kappa, nfields=10, npairs=200, steps=50, rsteps=0):
    """The network trained on the GPU at 32x16^3: nfields gauge fields x npairs
    sources (drawn on the device).  On every field, steps Adam steps on the
    imitation loss (targets M_sap source made by the library's SAP), then
    rsteps on the residual of one GCR step, |x - D N(x)|^2 / |x|^2; weights
    carried from field to field.  Returns (W, loss history, seconds, residual
    loss history)."""
    import numpy as np
    import torch
    chans = NET_CHANS
    nw = lqcd.Context.net_weight_count(chans)
    g = synth.gaussians(7, synth.STREAM_NET, 2 * nw)
    W = 0.02 * (g[0::2] + 1j * g[1::2])
    off = 0
    for l in range(len(chans) - 1):
        W[off:off + chans[l + 1] * chans[l] * 144].reshape(chans[l + 1], chans[l], 9, 4, 4)[0, 0, 0] += 0.7 * np.eye(4)
        off += chans[l + 1] * chans[l] * 144
    W = W.astype(np.complex64)
    tdims = (32, 16, 16, 16)
    hist, rhist, train_s = [], [], 0.0
    for f in range(nfields):
        c = lqcd.Context(tdims)
        c.set_gauge(torch.from_numpy(synth.su3_links(tdims, 100 + f)).cuda())
        c.clover_invert(kappa, CSW)
        gen = torch.Generator(device="cuda").manual_seed(1000 + f)
        src = torch.randn((npairs, c.V, 4, 3), dtype=torch.complex128, device="cuda", generator=gen)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c.net_set(chans, W, act=lqcd.BF16)
        h = c.net_train(src, steps=steps, batch=8, lr=2e-3, sap_prec=lqcd.F32)
        hr = c.net_train(src, steps=rsteps, batch=8, lr=1e-3, loss=lqcd.NET_LOSS_RESIDUAL) if rsteps else []
        torch.cuda.synchronize()
        train_s += time.perf_counter() - t0
        W = c.net_get()
        hist += [float(x) for x in h]
        rhist += [float(x) for x in hr]
        del src, c
    return W, hist, train_s, rhist


def run_net(args):
    """Learned preconditioner workload: a 3-layer parallel-transport network
    (1 -> 2 -> 2 -> 1 spinor fields, BF16, FP32 accumulation) trained on the GPU
    at 32x16^3 on 10 gauge fields x 200 sources (2000 pairs; targets M_sap
    source made by the library's SAP), then used at 64x32^3 (kappa = 0.1363)
    as the smoother of the deflated GCR, deflated SAP where its step fails.
    Reported beside the same deflated GCR with SAP, and plain SAP-GCR."""
    import numpy as np
    import torch
    from paper_1011_0911_gb300 import lqcd, synth
    kappa, chans = 0.1363, (1, 2, 2, 1)
    W, hist, train_s, rhist = train_net(lqcd, synth, kappa, args.nfields, args.npairs, args.train_steps,
                                        args.res_steps)
    dims = (64, 32, 32, 32)
    ctx = lqcd.Context(dims)
    ctx.set_gauge(torch.from_numpy(synth.su3_links(dims, 0)).cuda())
    ctx.clover_invert(kappa, CSW)
    ctx.net_set(chans, W, act=lqcd.BF16)
    eta = torch.from_numpy(synth.gaussian_spinor(ctx.Vh, 1)).cuda()
    Ns = 20
    v0 = torch.from_numpy(synth.gaussian_spinor(Ns * ctx.V, 100, synth.STREAM_SUBSPACE).reshape(Ns, ctx.V, 4, 3)).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.dfl_build(v0, bs=(4, 4, 4, 4), ninv=DFL_NINV, ncy=DFL_BUILD_SAP[0], nmr=DFL_BUILD_SAP[1], prec=lqcd.F32,
                  coarse_tol=1e-2, coarse_nmx=DFL_CNMX_EO if DFL_CEO else DFL_CNMX, coarse_nkv=DFL_CNKV,
                  coarse_prec=lqcd.F32, coarse_eo=DFL_CEO)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    out = {"mode": "net", "train_lattice": "32x16x16x16", "train_fields": args.nfields, "pairs": args.nfields * args.npairs,
           "train_steps": args.nfields * args.train_steps, "train_s": round(train_s, 3),
           "loss_first": round(float(np.mean(hist[:5])), 4), "loss_last": round(float(np.mean(hist[-5:])), 4),
           "residual_loss_last": round(float(np.mean(rhist[-5:])), 4) if rhist else None,
           "lattice": "64x32x32x32", "kappa": kappa, "subspace_build_s": round(build_s, 3)}
    forms = [("dfl_net", lqcd.SOLVER_DFL_NET_GCR), ("dfl_sap", lqcd.SOLVER_DFL_SAP_GCR), ("sap", lqcd.SOLVER_SAP_GCR)]
    for name, sid in forms:
        # the deflated forms take the time-to-solution table's SAP smoother, plain SAP-GCR its own 4 x 5
        sp = dict(ncy=DFL_SAP[0], nmr=DFL_SAP[1]) if sid != lqcd.SOLVER_SAP_GCR else dict(ncy=4, nmr=5)
        ctx.solve_dhat(eta, solver=sid, tol=1e-10, sap_prec=lqcd.F32, inner=lqcd.F32, check=False, **sp)   # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, info, st = ctx.solve_dhat(eta, solver=sid, tol=1e-10, sap_prec=lqcd.F32, inner=lqcd.F32, check=False, **sp)
        torch.cuda.synchronize()
        out[name] = {"seconds": round(time.perf_counter() - t0, 4), "iters": info[0]["iters"],
                     "net_fallbacks": info[0]["net_fallbacks"], "relres_dhat": info[0]["relres_dhat"], "status": st}
    out["gain_dfl_net_vs_dfl_sap"] = round(out["dfl_sap"]["seconds"] / out["dfl_net"]["seconds"], 3)
    print(json.dumps(out))


def run_netapply(args):
    """The network's three layers applied to 12 fields (the 12 sources of the
    deflated solve) at --lattice, BF16 activations, random weights: CUDA-event
    time per application and the layers' HBM roofline.  Algorithmic bytes of a
    layer per site and sample: every input channel read once (12 BF16 complex
    = 48 B), the eight links of the transports (2 rows FP32, 384 B, shared by
    the samples of a launch) and every output channel written once (48 B)."""
    import numpy as np
    import torch
    from paper_1011_0911_gb300 import lqcd, synth
    chans = NET_CHANS
    ctx = lqcd.Context(DIMS)
    ctx.set_gauge(torch.from_numpy(synth.su3_links(DIMS, 0)).cuda())
    nw = lqcd.Context.net_weight_count(chans)
    g = synth.gaussians(7, synth.STREAM_NET, 2 * nw)
    ctx.net_set(chans, (0.1 * (g[0::2] + 1j * g[1::2])).astype(np.complex64), act=lqcd.BF16)
    nb = args.nrhs
    x = torch.from_numpy(synth.gaussian_spinor(nb * ctx.V, 5).reshape(nb, ctx.V, 4, 3)).cuda()
    for _ in range(args.warmup):
        ctx.net_apply(x)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    for _ in range(args.steps):
        ctx.net_apply(x)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    V = ctx.V
    layer_bytes = sum(V * (nb * 48 * (ci + co) + 384) for ci, co in zip(chans[:-1], chans[1:]))
    peak, kind = load_peaks()
    print(json.dumps({"mode": "netapply", "lattice": "x".join(map(str, DIMS)), "fields": nb,
                      "ms_per_application": round(ms, 4), "layer_bytes_per_application": layer_bytes,
                      "layers_GBs_incl_conversions": round(layer_bytes / (ms * 1e-3) / 1e9, 1), "peak": peak,
                      "peak_kind": kind}))


def run_block(args):
    """DD-HMC block solves (Sec. 3): BiCGstab on every Dirichlet block of
    extents --bs (the paper's 6^2 x 12^2 at 48x24^3), one Gaussian source, FP64,
    tolerance 1e-10 per block.  One warm-up solve of two steps first.  The
    oracle's block operator is timed on the host cores for one application and
    scaled by the operator applications the GPU solve made (the oracle's solve
    itself takes minutes at this size)."""
    import torch
    import oracle as orc
    from paper_1011_0911_gb300 import lqcd, synth
    kappa = args.kappa or KAPPA_OF.get(DIMS, 0.1355)
    bs = tuple(int(v) for v in args.bs.split(","))
    U = synth.su3_links(DIMS, 0)
    ctx = lqcd.Context(DIMS)
    ctx.set_gauge(torch.from_numpy(U).cuda())
    ctx.clover_invert(kappa, CSW)
    eta_h = synth.gaussian_spinor(ctx.Vh, 1)
    eta = torch.from_numpy(eta_h).cuda()
    ctx.block_solve(eta, bs, tol=1e-10, nmx=2, check=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    psi, st, its, rr, sts = ctx.block_solve(eta, bs, tol=1e-10, nmx=1000, check=False)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    napp = 2 * int(its.max()) + 1   # lockstep: two block operators per step, one residual check
    out = {"mode": "block", "lattice": args.lattice, "kappa": kappa, "bs": list(bs), "nblk": int(len(its)),
           "status": int(st), "seconds": round(dt, 4), "iters_max": int(its.max()),
           "iters_mean": round(float(its.mean()), 1), "max_relres": float(rr.max()),
           "dhat_blk_applications": napp,
           "gflops": round(napp * FLOP_PER_SITE * ctx.Vh / dt / 1e9, 2)}
    if not args.no_cpu_baseline:
        o = orc.Oracle(DIMS, U, kappa, CSW)
        t0 = time.perf_counter()
        o.block_dhat(eta_h, bs)
        t1 = time.perf_counter() - t0
        out["cpu_baseline"] = {"kind": "oracle", "cores": orc.num_threads(),
                               "sample": "one application of the block operator on all blocks, scaled by the "
                                         "GPU solve's operator applications",
                               "seconds_per_application": round(t1, 3), "seconds_extrapolated": round(t1 * napp, 1)}
    print(json.dumps(out))


def run_configs(args):
    """The small configurations: Dhat per precision (one field, native
    resident, CUDA events) at 8^4 and 32x16^3, the 8^4 FP64 CGNR solve and the
    32x16^3 FP64 SAP-GCR solve to 1e-10 (plus the mixed forms), and the CPU
    oracle on the host cores: Dhat at both sizes, the 8^4 CGNR solve, and the
    32x16^3 SAP-GCR solve extrapolated from one SAP and one D application."""
    import torch
    import oracle as orc
    from paper_1011_0911_gb300 import lqcd, synth
    peak, peak_kind = load_peaks()
    out = {"mode": "configs", "hbm_peak_gbs": peak, "peak_kind": peak_kind, "oracle_threads": orc.num_threads()}
    for dims in ((8, 8, 8, 8), (32, 16, 16, 16)):
        kappa = KAPPA_OF[dims]
        U = synth.su3_links(dims, 0)
        ctx = lqcd.Context(dims)
        ctx.set_gauge(torch.from_numpy(U).cuda())
        ctx.clover_invert(kappa, CSW)
        tag = "x".join(map(str, dims))
        res = {"kappa": kappa, "dhat": {}}
        pe = synth.gaussian_spinor(ctx.Vh, 1)
        for name, prec in (("f64", lqcd.F64), ("f32", lqcd.F32), ("f16s", lqcd.F16S)):
            cdt = torch.complex128 if prec == lqcd.F64 else torch.complex64
            nin = ctx.pack(torch.from_numpy(pe).to(cdt).cuda(), prec, 1)
            nout = ctx.native_empty(prec, 1, 1)
            for _ in range(20):
                ctx.apply_Dhat_native(nin, nout, prec, 1)
            steps = 200
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(ctx.stream)
            for _ in range(steps):
                ctx.apply_Dhat_native(nin, nout, prec, 1)
            e1.record(ctx.stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / steps * 1e-3
            b = dhat_bytes_per_site(name, 1) * ctx.Vh
            res["dhat"][name] = {"us": round(t * 1e6, 2), "gflops": round(FLOP_PER_SITE * ctx.Vh / t / 1e9, 1),
                                 "hbm_frac_algorithmic": round(b / t / 1e9 / peak, 3),
                                 "note": "working set fits L2" if b < 100e6 else "working set exceeds L2"}
        o = orc.Oracle(dims, U, kappa, CSW)
        o.Dhat(pe)
        t0 = time.perf_counter()
        for _ in range(3):
            o.Dhat(pe)
        tc = (time.perf_counter() - t0) / 3
        res["oracle_dhat"] = {"seconds": round(tc, 5), "gflops": round(FLOP_PER_SITE * ctx.Vh / tc / 1e9, 3)}
        eta = torch.from_numpy(pe).cuda()
        if dims == (8, 8, 8, 8):
            ctx.solve_dhat(eta, solver=lqcd.SOLVER_CGNR, tol=1e-10, nmx=20000, check=False)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, info, st = ctx.solve_dhat(eta, solver=lqcd.SOLVER_CGNR, tol=1e-10, nmx=20000, check=False)
            torch.cuda.synchronize()
            res["cgnr_f64"] = {"seconds": round(time.perf_counter() - t0, 4), "iters": info[0]["iters"],
                               "relres_dhat": info[0]["relres_dhat"], "status": st}
            t0 = time.perf_counter()
            _, st, it = o.cgnr(pe, tol=1e-10)
            res["oracle_cgnr"] = {"seconds": round(time.perf_counter() - t0, 4), "iters": it, "status": st}
        forms = [("sap_gcr_f64", lqcd.F64, lqcd.F64), ("sap_gcr_f32", lqcd.F32, lqcd.F32),
                 ("sap_gcr_f16s", lqcd.F16S, lqcd.F32)]
        for name, sp, inner in forms:
            ctx.solve_dhat(eta, solver=lqcd.SOLVER_SAP_GCR, tol=1e-10, nmx=2, sap_prec=sp, inner=inner, check=False)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, info, st = ctx.solve_dhat(eta, solver=lqcd.SOLVER_SAP_GCR, tol=1e-10, sap_prec=sp, inner=inner,
                                         check=False)
            torch.cuda.synchronize()
            res[name] = {"seconds": round(time.perf_counter() - t0, 4), "iters": info[0]["iters"],
                         "relres_dhat": info[0]["relres_dhat"], "status": st}
        if dims == (32, 16, 16, 16):
            # Hasenbusch solve W(0.09) psi = eta (Eq. 3-4) beside the Dhat solve
            for name, sp, inner in (("hasenbusch_W_f64", lqcd.F64, lqcd.F64), ("hasenbusch_W_f32", lqcd.F32, lqcd.F32)):
                ctx.solve_W(eta, 0.09, tol=1e-10, nmx=2, sap_prec=sp, inner=inner, check=False)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, info, st = ctx.solve_W(eta, 0.09, tol=1e-10, sap_prec=sp, inner=inner, check=False)
                torch.cuda.synchronize()
                res[name] = {"dm": 0.09, "seconds": round(time.perf_counter() - t0, 4), "iters": info[0]["iters"],
                             "relres_W": info[0]["relres_dhat"], "status": st}
        full = synth.gaussian_spinor(ctx.V, 2)
        t0 = time.perf_counter()
        o.sap(full)
        t_sap = time.perf_counter() - t0
        t0 = time.perf_counter()
        o.D(full)
        t_d = time.perf_counter() - t0
        it = res["sap_gcr_f64"]["iters"]
        res["oracle_sap_gcr_estimate"] = {"seconds": round(it * (t_sap + t_d), 2), "sap_s": round(t_sap, 4),
                                          "d_s": round(t_d, 4),
                                          "sample": f"1 SAP + 1 D application, times the GPU's {it} GCR steps"}
        out[tag] = res
    print(json.dumps(out))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cb = cpu_baseline(steps=max(1, min(args.steps, 3)))
    line = {"impl": "reference", "metric": "Dhat GFLOP/s", "value": cb["value"], "unit": "GFLOP/s",
            "n_gpus": args.gpus, "steps": max(1, min(args.steps, 3)), "warmup": args.warmup,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (oracle: 1 field)", "lattice": "48x24x24x24"},
            "cpu_baseline": {k: cb[k] for k in ("kind", "cores", "sample")} | {"value": cb["value"], "unit": "GFLOP/s"},
            "e2e": {"value": cb["value"], "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nrhs", type=int, default=12)
    ap.add_argument("--prec", default="f32", choices=["f32", "f64", "f16s"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--no-solve", action="store_true", help="skip the time-to-solution comparison")
    ap.add_argument("--no-net", action="store_true", help="time-to-solution without the learned form")
    ap.add_argument("--lattice", default="48x24x24x24", help="TxL1xL2xL3 (profiling runs use smaller ones)")
    ap.add_argument("--mode", default="dhat", choices=["dhat", "solve", "batch", "net", "netapply", "configs", "block"],
                    help="solve: one time-to-solution run; batch: the uneven multi-lattice batch")
    ap.add_argument("--nlat", type=int, default=16, help="lattices of the batch mode")
    ap.add_argument("--nfields", type=int, default=10, help="net mode: training gauge fields")
    ap.add_argument("--npairs", type=int, default=200, help="net mode: sources per training field")
    ap.add_argument("--train-steps", type=int, default=50, help="net mode: Adam steps per training field")
    ap.add_argument("--res-steps", type=int, default=0,
                    help="Adam steps per training field on the GCR residual loss after the imitation steps "
                         "(a better one-step preconditioner, a worse deflated smoother: off by default)")
    ap.add_argument("--no-graph", action="store_true", help="batch mode: eager launches instead of graph replay")
    ap.add_argument("--solver", default="dfl", choices=["cgnr", "sap", "dfl"])
    ap.add_argument("--kappa", type=float, default=None)
    ap.add_argument("--Ns", type=int, default=20)
    ap.add_argument("--ninv", type=int, default=8)
    ap.add_argument("--ctol", type=float, default=1e-2)
    ap.add_argument("--cnmx", type=int, default=4096, help="iteration budget of each little-Dirac solve")
    ap.add_argument("--cnkv", type=int, default=16, help="Krylov vectors per little-Dirac GCR cycle (<= 32)")
    ap.add_argument("--cprec", default=None, choices=["f32", "f64"], help="little-Dirac operator precision")
    ap.add_argument("--krylov", default=None, choices=["f32", "f64"],
                    help="GCR Krylov-vector precision (f32 needs --prec f32)")
    ap.add_argument("--nkv", type=int, default=16, help="solve mode: GCR Krylov vectors per cycle")
    ap.add_argument("--bs", default="6,6,12,12", help="block mode: Dirichlet block extents")
    ap.add_argument("--ncy", type=int, default=4, help="solve mode: SAP cycles per preconditioner application")
    ap.add_argument("--nmr", type=int, default=5, help="solve mode: MinRes steps per SAP block solve")
    ap.add_argument("--bncy", type=int, default=4, help="solve mode: SAP cycles in the subspace build")
    ap.add_argument("--bnmr", type=int, default=4, help="solve mode: SAP MinRes steps in the subspace build")
    ap.add_argument("--bprec", default=None, choices=["f16s", "f32"],
                    help="solve mode: precision of the subspace build's SAP (default: the subspace's)")
    ap.add_argument("--ceo", action="store_true",
                    help="solve mode: even-odd (block-colour) form of the FP32 little-Dirac solve")
    ap.add_argument("--sap-prec", default=None, choices=["f16s", "f32", "f64"], help="solve mode: SAP precision")
    args = ap.parse_args()
    global DIMS
    DIMS = tuple(int(v) for v in args.lattice.split("x"))
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "solve":
        return run_solve(args)
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "net":
        return run_net(args)
    if args.mode == "configs":
        return run_configs(args)
    if args.mode == "netapply":
        return run_netapply(args)
    if args.mode == "block":
        return run_block(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_1011_0911_gb300 import lqcd, synth
    prec = {"f32": lqcd.F32, "f64": lqcd.F64, "f16s": lqcd.F16S}[args.prec]
    nrhs = args.nrhs
    U = synth.su3_links(DIMS, 0)
    ctx = lqcd.Context(DIMS)
    ctx.set_gauge(torch.from_numpy(U).cuda())
    ctx.clover_invert(KAPPA, CSW)
    Vh = ctx.Vh
    eta = synth.gaussian_spinor(nrhs * Vh, 1 + rank).reshape(nrhs, Vh, 4, 3)
    cdt = torch.complex128 if prec == lqcd.F64 else torch.complex64
    eta_host = torch.from_numpy(eta).to(cdt).pin_memory()
    eta_dev = eta_host.cuda()
    nin = ctx.pack(eta_dev, prec, 1)
    nout = ctx.native_empty(prec, 1, nrhs)
    stream = ctx.stream
    flops_step = FLOP_PER_SITE * Vh * nrhs

    # ---- device-resident timing (value, roofline)
    for _ in range(args.warmup):
        ctx.apply_Dhat_native(nin, nout, prec, nrhs)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    launches0 = ctx.kernel_launches
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    torch.cuda.synchronize()
    evs[0].record(stream)
    for i in range(args.steps):
        ctx.apply_Dhat_native(nin, nout, prec, nrhs)
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    launches = ctx.kernel_launches - launches0
    clk = clocks.stop()
    per = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    total_ms = max_over_ranks(evs[0].elapsed_time(evs[-1]), dist)
    ms_step = total_ms / args.steps
    value = whole_job_rate(flops_step, args.steps, world, total_ms) / 1e9
    avg_launch_ms = statistics.mean(per)
    bytes_app = dhat_bytes_per_site(args.prec, nrhs) * Vh
    peak, peak_kind = load_peaks()
    achieved = bytes_app / (avg_launch_ms * 1e-3) / 1e9

    # ---- end-to-end through the public ABI, host buffers, copies inside the timed region
    nbytes = eta_host.numel() * eta_host.element_size()
    e2e_ms, e2e_val = None, None
    if not args.no_e2e:
        out_host = torch.empty_like(eta_host).pin_memory()
        e2e_steps = max(3, min(args.steps // 10, 40))
        for _ in range(2):
            d = eta_host.to("cuda", non_blocking=True)
            o = ctx.apply_Dhat(d, prec)
            out_host.copy_(o, non_blocking=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(e2e_steps):
            d = eta_host.to("cuda", non_blocking=True)
            o = ctx.apply_Dhat(d, prec)
            out_host.copy_(o, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(e0.elapsed_time(e1), dist) / e2e_steps
        e2e_val = round(whole_job_rate(flops_step, 1, world, e2e_ms) / 1e9, 2)
        e2e_ms = round(e2e_ms, 4)

    tts = None
    # the time-to-solution table (minutes of GPU time) belongs to the one-GPU run;
    # under torchrun the other GPUs would idle meanwhile
    if not args.no_solve and world == 1 and DIMS == (48, 24, 24, 24):
        net = None
        if not args.no_net:
            W, hist, train_s, rhist = train_net(lqcd, synth, KAPPA, args.nfields, args.npairs, args.train_steps,
                                                args.res_steps)
            net = {"W": W, "pairs": args.nfields * args.npairs, "train_s": round(train_s, 3),
                   "loss_first": round(sum(hist[:5]) / 5, 4), "loss_last": round(sum(hist[-5:]) / 5, 4),
                   "residual_loss_last": round(sum(rhist[-5:]) / 5, 4) if rhist else None}
        tts = time_to_solve(ctx, lqcd, eta_dev.to(torch.complex128), net)

    if rank == 0:
        cb = None
        if not args.no_cpu_baseline:
            cb = cpu_baseline()
        line = {
            "metric": "Dhat GFLOP/s", "value": round(value, 2), "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.prec, "data": "synthetic",
            "config": {"workload": WORKLOAD, "lattice": args.lattice, "nrhs": nrhs, "precision": args.prec,
                       "links": {lqcd.F32: "2-row SU(3)", lqcd.F64: "full SU(3)",
                                 lqcd.F16S: "2-row SU(3) FP16, FP16 clover"}[prec],
                       "l2": "inputs larger than L2 (links+clover+12 fields = %.2f GB)" % (
                           (dhat_bytes_per_site(args.prec, nrhs) * Vh) / 1e9),
                       "parallelism": f"replicas x{world}"},
            "e2e": {"value": e2e_val, "unit": "GFLOP/s", "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                    "path": "lqcd_apply_Dhat (canonical fields) + pinned host copies"},
            "roofline": {"kernel": "Dhat = DHAT1 + DHAT2 stencil kernels (k_hop / k_hop_mr, form and shape chosen by the autotuner)", "bound": "hbm",
                         "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                         "traffic": traffic_of(args.prec, nrhs, Vh),
                         "traffic_source": TRAFFIC_NOTE if traffic_of(args.prec, nrhs, Vh) else None,
                         "algorithmic_bytes_per_launch": bytes_app},
            "gpu_launches": launches,
            "clocks": clk,
            "cpu_baseline": cb,
            "time_to_solve": tts,
        }
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
