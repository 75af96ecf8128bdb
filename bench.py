"""Benchmark of the HQMC hot path: HMC trajectories per second on one GB300.

A step is one HMC trajectory of the whole path (Philox draws, phi = M^dagger R,
N_lf + 1 CG solves of (M^dagger M) X = phi, forces, leapfrog, Metropolis) on a
seeded synthetic gauge field; the chain continues from step to step.

Default workload (learned + mixed precision against plain FP64): L = 66,
Ntau = 660 (2,874,960 sites), dtau = 0.1, t = 1, J = 1, compact action, CG to a
true FP64 residual of 1e-8, 20 leapfrog steps.  Untimed set-up: from the cold
start (pi flux + N(0, 0.3^2) per bond, tau-independent, random gauge
transformation) the chain is thermalised with the preconditioned mixed solver
for up to 400 trajectories (200 s) while dt follows the acceptance (grown x1.25 after 4
accepted trajectories in a row, shrunk x0.8 when 2 or fewer of 4 were accepted);
dt is then frozen where <dH> (~ dt^4) of the last 40 trajectories
predicts <dH> = 0.1, i.e. an acceptance near 0.8.  Then 8 more trajectories give
32 (theta, phi, x) triples (4 sources each) and the net takes 8 Adam epochs over
them.  The timed steps use the learned solver; the same chain state is then
advanced with plain FP64 CG and with the factor arms (pcg64, mixed, pmixed) on
the same draws, dt, N_lf and tolerance, and the fused M^dagger M apply is timed
alone with L2 flushed.

Workload hmc_fp64_L24_Nt240 (plain FP64 GPU HMC): L = 24, Ntau = 240 (138,240
sites), CG to 1e-8, 20 leapfrog steps of dt = 0.0005.  Start (inputs.theta_ordered with tau_walk=0):
the pi-flux background favoured by half-filled fermions plus N(0, 0.3^2) on every
bond, the same at every tau, under a random gauge transformation.  A start
i.i.d. on every bond and slice makes M^dagger M so singular at this size that
FP64 CG needs more than 6e4 iterations per solve, and fields that wander in tau
let the pseudofermion force drive the leapfrog into singular configurations.
The step keeps |dH| below 1 at this volume (|dH| grows like volume * dt^2 from
a cold start: 125 at dt = 0.01, 31 at dt = 0.005, measured).

Workload estimate_L66_Nt660_40rv (stochastic estimation): a step is one estimate
of diag M^{-1} with 40 CN(0, 1) vectors on one L = 66 field (pmixed to 1e-8),
solved one after another (the line's value), with projected initial guesses
(`projected`) and with the 40 systems advancing together (`together`, whose
multi-system walk launch is the line's roofline).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

Prints one JSON line on rank 0.  Under torchrun every rank runs an independent
chain (replicas; the path has no exchange between chains).  --impl reference
times the FP64 CPU oracle on the host cores on a bounded sample of the same
workload.
"""
from __future__ import annotations

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

METRIC = "M†M apply GB/s vs HBM peak; HMC traj/s learned+FP32 vs plain FP64 at 1e-8"

WORKLOADS = {
    # plain FP64 HMC at L = 24, Ntau = 240
    "hmc_fp64_L24_Nt240": dict(L=24, Ntau=240, dtau=0.1, t=1.0, J=1.0, nsteps=20, dt=0.0005, tol=1e-8,
                               solver="cg64", seed=1, start="cold"),
    # plain FP64 HMC at L = 8, Ntau = 40 (oracle-sized)
    "hmc_fp64_L8_Nt40": dict(L=8, Ntau=40, dtau=0.1, t=1.0, J=1.0, nsteps=10, dt=0.02, tol=1e-10,
                             solver="cg64", seed=1, start="hot"),
    # mixed precision at L = 48, Ntau = 480
    "hmc_mixed_L48_Nt480": dict(L=48, Ntau=480, dtau=0.1, t=1.0, J=1.0, nsteps=20, dt=0.00018, tol=1e-8,
                                solver="mixed", seed=1, start="cold"),
}
# batched chains: 32 lattices, L in {12, 16, 20, 24} x 8, Ntau = 10 L, one trajectory of every chain per step
BATCH_LATTICES = [(L, 10 * L) for L in (12, 16, 20, 24) for _ in range(8)]
WORKLOADS["batched_32chains_L12-24"] = dict(L=24, Ntau=240, dtau=0.1, t=1.0, J=1.0, nsteps=20, dt=0.0005, tol=1e-8,
                                            solver="cg64", seed=100, start="cold", batched=True)
# the same batch with the tau-line preconditioner in the batched CG (FP64)
WORKLOADS["batched_32chains_L12-24_pcg64"] = dict(WORKLOADS["batched_32chains_L12-24"], solver="pcg64")
# learned + mixed precision at L = 66, Ntau = 660 against plain FP64 on the same chain state.  Untimed
# set-up: from the cold start the chain is thermalised with the preconditioned mixed solver while dt is
# adapted to the acceptance (the Methods tune dt adaptively); dt is then frozen.  The net is trained on
# (theta, phi, x) triples the sampler produces at this size.  The timed steps use that dt.
WORKLOADS["hmc_learned_fp32_L66_Nt660"] = dict(L=66, Ntau=660, dtau=0.1, t=1.0, J=1.0, nsteps=20, dt=2e-4,
                                               tol=1e-8, solver="plearned", seed=1, start="cold",
                                               therm=400, therm_s=200.0,
                                               compare="cg64", compare_steps=5, factors=("pcg64", "mixed", "pmixed", "flearned"),
                                               factor_steps=3, triple_trajs=8, rhs_per_traj=4, epochs=8,
                                               lr=1e-3, guess=4)
# stochastic estimation (Methods): 40 CN(0,1) vectors on one field, M^{-1} xi by preconditioned mixed CG
WORKLOADS["estimate_L66_Nt660_40rv"] = dict(L=66, Ntau=660, dtau=0.1, t=1.0, J=1.0, nsteps=0, dt=0.0, tol=1e-8,
                                            solver="pmixed", seed=1, start="cold", estimate=True, nrv=40)
DEFAULT_WORKLOAD = "hmc_learned_fp32_L66_Nt660"

# Algorithmic work of one launch of the fused M^dagger M kernel in CG mode, per site:
#   flops: 2 sweeps x 7 factor passes x 8 flops + 22 (direction update, combination, <p, Op>)
#   bytes (FP64): links 32 + r 16 + p_old 16 + p_new 16 + q 16
#   bytes (FP32, register-blocked): theta as float 8 + r 8 + p_old 8 + p_new 8 + q 8
MDAGM_FLOPS_PER_SITE = 134
MDAGM_BYTES_PER_SITE = {"cg64": 96, "pcg64": 96, "mixed": 40, "learned": 40, "pmixed": 40, "plearned": 40}


# DRAM bytes (read + write) of one launch of the dominant kernel from an ncu capture of the τ-walking
# FP32 kernel at L = 66 (cold caches; writes still in L2 at the kernel's end are not counted there).
# Valid for the kernel as captured; set to None when the kernel changes.
NCU_TRAFFIC_BYTES = {"hmc_learned_fp32_L66_Nt660": 79.50208e6 + 9.959936e6}


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest x over the ranks: a job's time is that of its slowest replica."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: every replica's units over the slowest replica's time."""
    return world * units_per_rank / seconds


def rank_seed(seed: int, rank: int) -> int:
    """Each replica runs its own chain, with seeds 1000 apart."""
    return seed + 1000 * rank


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", self.gpu_id], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample(wl: dict, its_per_traj: float, theta, phi, max_iters: int = 10):
    """Times the FP64 CPU oracle on a bounded sample of one trajectory: max_iters
    iterations of the workload's CG (preconditioned with the oracle's tau-line
    preconditioner when the workload's solver is) and one force evaluation at the
    workload's size, scaled to one trajectory with its_per_traj CG iterations and
    nsteps + 1 forces."""
    import oracle
    from oracle import precond as opc

    lat = oracle.Lattice(wl["L"], wl["Ntau"], dtau=wl["dtau"], t=wl["t"], J=wl["J"])
    pc = wl["solver"].startswith("p")
    t0 = time.perf_counter()
    if pc:
        X, it, _ = opc.pcg(lat, theta, phi, opc.coefficients(lat), tol=1e-30, maxit=max_iters)
    else:
        X, it, _, _ = oracle.cg(lat, theta, phi, tol=1e-30, maxit=max_iters)
    t1 = time.perf_counter()
    oracle.fermion_dS(lat, theta, X)
    oracle.bosonic_dS(lat, theta)
    t2 = time.perf_counter()
    t_iter = (t1 - t0) / (it + 2)  # it iterations plus the initial and final residual applications
    t_force = t2 - t1
    t_traj = its_per_traj * t_iter + (wl["nsteps"] + 1) * t_force
    kind = "preconditioned CG" if pc else "CG"
    return {"traj_s": t_traj, "t_iter_s": t_iter, "t_force_s": t_force, "cores": oracle.num_threads(),
            "sample_s": t2 - t0,
            "sample": f"{it} oracle {kind} iterations + 1 force at L={wl['L']}, Ntau={wl['Ntau']}, "
                      f"scaled to {its_per_traj:.0f} iterations and {wl['nsteps'] + 1} forces per trajectory"}


# CG iterations per trajectory used to scale oracle samples when no GPU run is
# available (the reference arm); measured on the GPU with the same algorithm.
ITS_PER_TRAJ_HINT = {"hmc_fp64_L24_Nt240": 11000.0, "hmc_fp64_L8_Nt40": 6000.0, "hmc_mixed_L48_Nt480": 16500.0,
                     "batched_32chains_L12-24": 11000.0, "batched_32chains_L12-24_pcg64": 1800.0,
                     "hmc_learned_fp32_L66_Nt660": 2950.0,
                     "estimate_L66_Nt660_40rv": 250.0}
# oracle CG iterations per bounded sample (the largest lattices take about a second per iteration on the host)
ORACLE_SAMPLE_ITERS = {"hmc_learned_fp32_L66_Nt660": 4, "hmc_mixed_L48_Nt480": 6, "estimate_L66_Nt660_40rv": 4}


def run_reference(args, wl_name, wl, rank, world):
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_2508_16298_gb300 import inputs

    lat = oracle.Lattice(wl["L"], wl["Ntau"], dtau=wl["dtau"], t=wl["t"], J=wl["J"])
    theta = start_theta(wl, wl["seed"])
    R = inputs.complex_gaussian(wl["L"], wl["Ntau"], wl["seed"] + 1)
    phi = oracle.apply_M(lat, theta, R, dagger=True)
    its = ITS_PER_TRAJ_HINT[wl_name]
    n_it = ORACLE_SAMPLE_ITERS.get(wl_name, 10)
    unit = "traj/s"
    if wl.get("estimate"):  # a unit of work is one random vector: its solve, no force
        wl = dict(wl, nsteps=-1)
        unit = "random vectors/s"
    for _ in range(args.warmup):
        oracle_sample(wl, its, theta, phi, max_iters=1)
    samples = [oracle_sample(wl, its, theta, phi, max_iters=n_it) for _ in range(args.steps)]
    t = statistics.median(s["traj_s"] for s in samples)
    value = 1.0 / t
    # a step is one bounded sample: ms_per_step is its wall time, and the rate is the
    # fraction of a trajectory it covers over that time (= 1 / extrapolated seconds per trajectory)
    sample_s = statistics.median(s["sample_s"] for s in samples)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": unit, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sample_s,
            "work_per_step": {"fraction_of_unit": sample_s / t, "extrapolated_s_per_unit": t,
                              "value": "fraction_of_unit / (ms_per_step / 1000)"},
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(wl_name, WORKLOADS[wl_name]),
            "cpu_baseline": {"value": value, "unit": unit, "cores": samples[0]["cores"], "kind": "oracle",
                             "sample": samples[0]["sample"]},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def start_theta(wl, seed):
    from paper_2508_16298_gb300 import inputs
    if wl["start"] == "hot":
        return inputs.theta_hot(wl["L"], wl["Ntau"], seed)
    if wl["start"] == "ordered":
        return inputs.theta_ordered(wl["L"], wl["Ntau"], seed, J=wl["J"], dtau=wl["dtau"])
    if wl["start"] == "cold":
        return inputs.theta_ordered(wl["L"], wl["Ntau"], seed, J=wl["J"], dtau=wl["dtau"], tau_walk=0.0)
    return inputs.theta_warm(wl["L"], wl["Ntau"], seed, J=wl["J"], dtau=wl["dtau"])


SOLVER_TEXT = {
    "cg64": "cg64: FP64 CG",
    "pcg64": "pcg64: FP64 CG preconditioned with the tau-line preconditioner",
    "mixed": "mixed: FP32 M^dagger M in CG, FP64 reliable updates every 50 iterations",
    "pmixed": "pmixed: the mixed solver preconditioned with the tau-line preconditioner (FP32)",
    "learned": "learned: net-corrected initial guess (kept if it lowers the FP32 residual norm; with the chronological guess "
               "tried until two tries in an integration fail to halve it), then the mixed solver",
    "plearned": "plearned: net-corrected initial guess (kept if it lowers the FP32 residual norm; with the chronological guess "
                "tried until two tries in an integration fail to halve it), then the mixed solver preconditioned with the "
                "tau-line preconditioner (FP32)",
    "flearned": "flearned: net-corrected initial guess, then flexible CG (Polak-Ribiere beta) with the net as preconditioner "
                "every iteration, FP32 recurrence with FP64 reliable updates, tau-line pmixed as the fallback",
}


def config_of(wl_name, wl):
    return {"workload": wl_name, "L": wl["L"], "Ntau": wl["Ntau"], "sites": wl["L"] * wl["L"] * wl["Ntau"],
            "dtau": wl["dtau"], "t": wl["t"], "J": wl["J"], "action": "compact",
            "start": {"hot": "hot: theta i.i.d. U[-pi, pi)",
                      "warm": "warm: U[-pi, pi) per bond + periodic Gaussian walk in tau, step var J*dtau/2",
                      "ordered": "pi-flux + N(0, 0.3^2) per bond + periodic Gaussian walk in tau (step var "
                                 "J*dtau/2) + random gauge transformation",
                      "cold": "pi-flux + N(0, 0.3^2) per bond, tau-independent, + random gauge transformation"}
                     [wl["start"]],
            "n_leapfrog": wl["nsteps"],
            "dt": (f"adapted to the acceptance during {wl['therm']} untimed thermalisation trajectories from "
                   f"{wl['dt']}, then frozen (value in the line's dt)") if wl.get("therm") else wl["dt"],
            "cg_tol": wl["tol"],
            "solver": SOLVER_TEXT[wl["solver"]],
            "initial_guess": (f"chronological: each leapfrog solve after the first starts from the Galerkin solution "
                              f"in the span of the last {wl['guess']} solutions of the integration (O in FP32)")
                             if wl.get("guess") else "the previous solution of the integration",
            "l2": "flushed between timed steps (512 MiB write; step times exclude the flush)"}


def kernel_name(shape, prec):
    v = shape["variant"]
    if v >= 100:
        return f"mdagm_walk_kernel<{prec}, CG direction, nby={v - 100}> (tau-walking, {shape['threads']} threads)"
    if v > 0:
        return f"mdagm_block_kernel<{prec}, CG direction, nby={v}> (cluster {shape['cluster']})"
    return f"mdagm_kernel<{prec}, CG direction, mb={-v}> (cluster {shape['cluster']})"


THERM_COUNTER = 10 ** 5   # Philox trajectory counters of the thermalisation
TRIPLE_COUNTER = 10 ** 6  # ... of the trajectories that produce training triples


def thermalize(hqmc, cfg, theta, wl, seed):
    """Untimed set-up: from the start field, trajectories with the preconditioned mixed
    solver while dt follows the acceptance (the Methods tune dt adaptively): after every
    4 trajectories dt grows by 1.25 if all 4 were accepted and shrinks by 0.8 if 2 or
    fewer were, which holds the acceptance near 0.75-0.9.  Stops after `therm`
    trajectories or `therm_s` seconds; the last dt is the production dt.  Returns
    (dt, report) with the bosonic action S_B and the CG iterations over the run, so
    that their levelling off can be read."""
    dt = wl["dt"]
    rows, window = [], []
    hqmc.set_guess_history(cfg, wl.get("guess", 0))
    t0 = time.perf_counter()
    k = 0
    while k < wl["therm"] and time.perf_counter() - t0 < wl["therm_s"]:
        sb = hqmc.action_terms(cfg, theta)[0]
        inf = hqmc.trajectory(cfg, theta, seed=seed, traj_counter=THERM_COUNTER + k, nsteps=wl["nsteps"], dt=dt,
                              tol=wl["tol"], solver="pmixed")
        rows.append((dt, inf["accepted"], inf["cg_iterations"], sb, inf["dH"]))
        window.append(inf["accepted"])
        k += 1
        if len(window) == 4:
            acc = sum(window)
            dt = dt * 1.25 if acc == 4 else dt * 0.8 if acc <= 2 else dt
            window = []
    n = len(rows)
    tenth = max(1, n // 10)
    last = rows[-min(n, 40):]
    # production dt: at fixed N_lf the leapfrog's <dH> grows like dt^4; the last 40
    # trajectories, each rescaled to the controller's final dt, estimate <dH> there,
    # and dt is set where <dH> = 0.1 (acceptance erfc(sqrt(<dH>)/2) = 0.82), within
    # [0.7, 1.15] x the final dt
    m = statistics.mean(r[4] * (dt / r[0]) ** 4 for r in last)
    dt_prod = dt * min(1.15, max(0.7, (0.1 / max(m, 1e-3)) ** 0.25))
    report = {"trajectories": n, "seconds": round(time.perf_counter() - t0, 1), "solver": "pmixed",
              "dt_first": rows[0][0], "dt_controller_final": dt, "mean_dH_last_40_at_that_dt": m,
              "dt_production": dt_prod,
              "rule": "every 4 trajectories: dt x1.25 if 4 accepted, x0.8 if <= 2 accepted; production dt from "
                      "<dH> ~ dt^4 over the last 40, aiming at <dH> = 0.1",
              "S_B_per_bond": {"first": rows[0][3] / (2 * cfg.n_sites),
                               "mean_prev_tenth": statistics.mean(r[3] for r in rows[-2 * tenth:-tenth]) / (2 * cfg.n_sites)
                               if n >= 2 * tenth + 1 else None,
                               "mean_last_tenth": statistics.mean(r[3] for r in rows[-tenth:]) / (2 * cfg.n_sites)},
              "cg_iterations_per_traj": {"first_tenth": statistics.mean(r[2] for r in rows[:tenth]),
                                         "prev_tenth": statistics.mean(r[2] for r in rows[-2 * tenth:-tenth])
                                         if n >= 2 * tenth + 1 else None,
                                         "last_tenth": statistics.mean(r[2] for r in rows[-tenth:])},
              "acceptance_last_40": statistics.mean(r[1] for r in last)}
    return dt_prod, report


def train_net_streamed(hqmc, inputs, cfg, wl, theta, dt, seed, dev):
    """Online training on wl["train_triples"] sampler triples that are never stored:
    the chain advances one trajectory at the production dt, then `stream_sources`
    sources phi = M^dagger R on that field are solved (preconditioned mixed CG,
    FP64 residual 1e-8) and each (theta, phi, x) takes one Adam step as soon as it
    exists.  Device memory stays that of one triple, whatever the count.  Returns
    the net and a report with the mean loss over each block of 100 triples."""
    import torch
    L, N = wl["L"], wl["Ntau"]
    total, per = wl["train_triples"], wl["stream_sources"]
    kw = dict(nsteps=wl["nsteps"], dt=dt, tol=wl["tol"], solver="pmixed")
    net = hqmc.Net(seed=seed)
    hqmc.set_preconditioner(cfg, net)
    losses, curve = [], []
    t_sample = t_train = 0.0
    k = 0
    while len(losses) < total:
        t0 = time.perf_counter()
        hqmc.trajectory(cfg, theta, seed=seed, traj_counter=TRIPLE_COUNTER + k, **kw)
        for m in range(min(per, total - len(losses))):
            R = torch.from_numpy(inputs.complex_gaussian(L, N, seed * 7919 + 97 * k + m)).to(dev)
            phi = hqmc.apply_M(cfg, theta, R, dagger=True)
            x, _ = hqmc.cg_solve(cfg, theta, phi, tol=wl["tol"], solver="pmixed")
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            t_sample += t1 - t0
            losses.append(net.train_step(cfg, theta, phi, x, lr=wl["lr"]))
            t0 = time.perf_counter()
            t_train += t0 - t1
            if len(losses) % 100 == 0:
                curve.append(round(statistics.mean(losses[-100:]), 4))
        k += 1
    return net, {"triples": len(losses), "stored": 0, "trajectories": k, "sources_per_trajectory": per,
                 "epochs": 1, "sampler_s": round(t_sample, 2), "train_s": round(t_train, 2),
                 "loss_per_100_triples": curve, "loss": "||K(theta) phi - x||^2 / ||x||^2"}


def train_net(hqmc, inputs, cfg, wl, theta, dt, seed, dev):
    """Untimed set-up of the learned solver: `triple_trajs` trajectories of the chain at the
    production dt; after each, `rhs_per_traj` sources phi = M^dagger R with fresh Gaussian R
    and x = (M^dagger M)^{-1} phi (preconditioned mixed CG, FP64 residual 1e-8) form
    training triples (theta, phi, x).  The net then takes `epochs` Adam passes over them.
    Returns the net and a report with the loss per epoch."""
    import torch
    L, N = wl["L"], wl["Ntau"]
    kw = dict(nsteps=wl["nsteps"], dt=dt, tol=wl["tol"], solver="pmixed")
    trips = []
    t0 = time.perf_counter()
    for k in range(wl["triple_trajs"]):
        hqmc.trajectory(cfg, theta, seed=seed, traj_counter=TRIPLE_COUNTER + k, **kw)
        th = theta.clone()
        for m in range(wl["rhs_per_traj"]):
            R = torch.from_numpy(inputs.complex_gaussian(L, N, seed * 7919 + 97 * k + m)).to(dev)
            phi = hqmc.apply_M(cfg, th, R, dagger=True)
            x, _ = hqmc.cg_solve(cfg, th, phi, tol=wl["tol"], solver="pmixed")
            trips.append((th, phi, x))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    net = hqmc.Net(seed=seed)
    hqmc.set_preconditioner(cfg, net)  # allocates the config's net workspace
    curve = []
    for ep in range(wl["epochs"]):
        losses = [net.train_step(cfg, th, ph, x, lr=wl["lr"]) for th, ph, x in trips]
        curve.append(round(statistics.mean(losses), 4))
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    return net, {"triples": len(trips), "trajectories": wl["triple_trajs"], "sources_per_trajectory": wl["rhs_per_traj"],
                 "epochs": wl["epochs"], "sampler_s": round(t1 - t0, 2), "train_s": round(t2 - t1, 2),
                 "loss_per_epoch": curve, "loss": "||K(theta) phi - x||^2 / ||x||^2"}


def same_draws_arm(hqmc, cfg, theta_start, seed, first_counter, n, solver, wl, dt, flush, stream, guess=0):
    """The chain advanced from theta_start with `solver` on the draws of the first n timed
    steps (counters first_counter ...), dt, N_lf and tolerance unchanged; one untimed
    single-solve trajectory first builds the solver's CUDA graph.  guess: the
    chronological guess history of the arm (0: the previous solution).  Returns
    per-step data; the config's guess setting is restored to the workload's."""
    import torch
    hqmc.set_guess_history(cfg, guess)
    th = theta_start.clone()
    kw = dict(nsteps=wl["nsteps"], dt=dt, tol=wl["tol"], solver=solver)
    hqmc.trajectory(cfg, th.clone(), seed=seed, traj_counter=first_counter, **dict(kw, nsteps=0))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    infos = []
    for k in range(n):
        flush.zero_()
        ev[k][0].record(stream)
        infos.append(hqmc.trajectory(cfg, th, seed=seed, traj_counter=first_counter + k, **kw))
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    hqmc.set_guess_history(cfg, wl.get("guess", 0))
    ms = [a.elapsed_time(b) for a, b in ev]
    return {"solver": solver, "guess_history": guess, "traj_per_s": n / (sum(ms) / 1e3), "steps": n,
            "acceptance": statistics.mean(i["accepted"] for i in infos),
            "accepted": [i["accepted"] for i in infos],
            "cg_iterations_per_traj": statistics.mean(i["cg_iterations"] for i in infos),
            "dH": [round(i["dH"], 6) for i in infos],
            "max_true_residual": max(i["max_true_residual"] for i in infos),
            "step_ms": [round(m, 3) for m in ms]}


def time_apply(hqmc, cfg, theta, x, flush, timer, reps=20):
    """Average device time of the fused M^dagger M kernel alone (library event timer)
    over reps applies, L2 flushed before each."""
    import torch
    y = torch.empty_like(x)
    hqmc.apply_MdagM(cfg, theta, x, y=y)
    hqmc.set_timing(cfg, True)
    hqmc.get_timing(cfg, timer)
    for k in range(reps):
        flush.fill_(float(k))
        hqmc.apply_MdagM(cfg, theta, x, y=y)
    n, ms = hqmc.get_timing(cfg, timer)
    hqmc.set_timing(cfg, False)
    return 1e3 * ms / max(n, 1)


def run_ours(args, wl_name, wl, rank, world, local_rank):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_16298_gb300 import hqmc, inputs

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    L, N = wl["L"], wl["Ntau"]
    sites = L * L * N
    cfg = hqmc.Config(L, N, dtau=wl["dtau"], t=wl["t"], J=wl["J"], autotune=True)
    seed = rank_seed(wl["seed"], rank)
    theta = torch.from_numpy(start_theta(wl, seed)).to(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    therm = None
    dt = wl["dt"]
    if wl.get("therm"):
        dt, therm = thermalize(hqmc, cfg, theta, wl, seed)
    kw = dict(nsteps=wl["nsteps"], dt=dt, tol=wl["tol"], solver=wl["solver"])
    learned = None
    net = None
    if wl["solver"] in ("learned", "plearned"):
        trainer = train_net_streamed if wl.get("train_triples") else train_net
        net, learned = trainer(hqmc, inputs, cfg, wl, theta, dt, seed, dev)

    for k in range(args.warmup):
        hqmc.trajectory(cfg, theta, seed=seed, traj_counter=k, **kw)
    fp64_tflops = hqmc.probe_fp64_rate(cfg) if rank == 0 else None
    theta_start = theta.clone()  # chain state at the start of the timed region (for the FP64 arm)

    # ---- device-resident timed region --------------------------------------
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    infos = []
    try:
        props = torch.cuda.get_device_properties(dev)
        gpu_id = "GPU-" + str(props.uuid) if getattr(props, "uuid", None) else str(local_rank)
    except Exception:
        gpu_id = str(local_rank)
    clocks = ClockSampler(gpu_id)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = cfg.launch_count()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        infos.append(hqmc.trajectory(cfg, theta, seed=seed, traj_counter=args.warmup + k, **kw))
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    launches = cfg.launch_count() - launches0
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)

    # ---- dominant kernel: CUDA events around every launch of the fused M^dagger M
    # during one more trajectory (event timing runs the CG loop bodies from the
    # host, since per-launch events cannot sit inside the device-side loop) ----
    fp32 = wl["solver"] not in ("cg64", "pcg64")
    flush.zero_()
    hqmc.set_timing(cfg, True)
    hqmc.trajectory(cfg, theta, seed=seed, traj_counter=args.warmup + args.steps, **kw)
    n_md, md_ms = hqmc.get_timing(cfg, hqmc.TIMER_MDAGM32 if fp32 else hqmc.TIMER_MDAGM)
    n_up, up_ms = hqmc.get_timing(cfg, hqmc.TIMER_CG_UPDATE)
    n_pc, pc_ms = hqmc.get_timing(cfg, hqmc.TIMER_PRECOND)
    # per-launch times: a loop body's launches after its solve converged exit at once, so
    # the median (not the mean) is the time of a launch that does the work
    md_us = hqmc.get_timing_samples(cfg, hqmc.TIMER_MDAGM32 if fp32 else hqmc.TIMER_MDAGM)
    up_us = hqmc.get_timing_samples(cfg, hqmc.TIMER_CG_UPDATE)
    pc_us = hqmc.get_timing_samples(cfg, hqmc.TIMER_PRECOND)
    hqmc.set_timing(cfg, False)
    total_ms = max_over_ranks(total_ms, world, dev)
    value = job_rate(args.steps, world, total_ms / 1e3)

    # ---- end to end through the public API with host buffers ----------------
    theta_h = theta.cpu().pin_memory()
    bytes_theta = theta_h.numel() * 8
    e2e_steps = min(5, args.steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        th_dev = theta_h.to(dev, non_blocking=True)
        hqmc.trajectory(cfg, th_dev, seed=seed, traj_counter=args.warmup + args.steps + 1 + k, **kw)
        theta_h.copy_(th_dev, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, world, dev)
    e2e_value = job_rate(e2e_steps, world, e2e_s)

    # ---- other solvers on the same chain state and draws (dt, N_lf, tolerance unchanged) -----
    compare, factors = None, None
    if wl.get("compare"):
        n64 = min(wl.get("compare_steps", 5), args.steps)
        compare = same_draws_arm(hqmc, cfg, theta_start, seed, args.warmup, n64, wl["compare"], wl, dt, flush, stream)
        ours = sum(step_ms[:n64]) / 1e3
        compare["speedup_same_draws"] = (sum(compare["step_ms"]) / 1e3) / ours
        compare["speedup"] = (value / world) / compare["traj_per_s"]
        compare["same_draws_as_steps"] = list(range(n64))
        compare["dH_difference_max"] = max(abs(a - b["dH"]) for a, b in zip(compare["dH"], infos[:n64]))
        compare["same_accept_decisions"] = all(a == b["accepted"] for a, b in zip(compare["accepted"], infos[:n64]))
    if wl.get("factors"):
        nf = min(wl.get("factor_steps", 3), args.steps)
        g = wl.get("guess", 0)
        arms = {sv: same_draws_arm(hqmc, cfg, theta_start, seed, args.warmup, nf, sv, wl, dt, flush, stream, g)
                for sv in wl["factors"]}
        if g:  # the same solver without the chronological guess
            arms["pmixed_previous_guess"] = same_draws_arm(hqmc, cfg, theta_start, seed, args.warmup, nf, "pmixed",
                                                           wl, dt, flush, stream, 0)
        t = {sv: sum(a["step_ms"]) for sv, a in arms.items()}
        t[wl["solver"]] = sum(step_ms[:nf])
        factors = {"steps": nf, "ms_same_draws": {k: round(v, 1) for k, v in t.items()},
                   "its_per_traj": {sv: a["cg_iterations_per_traj"] for sv, a in arms.items()},
                   "fp32_over_fp64": t["pcg64"] / t["pmixed"] if "pcg64" in t and "pmixed" in t else None,
                   "precond_gain": t["mixed"] / t["pmixed"] if "mixed" in t and "pmixed" in t else None,
                   "net_gain": t["pmixed"] / t[wl["solver"]] if "pmixed" in t else None,
                   "fcg_net_gain": t["pmixed"] / t["flearned"] if "flearned" in t and "pmixed" in t else None,
                   "guess_gain": t["pmixed_previous_guess"] / t["pmixed"] if "pmixed_previous_guess" in t else None,
                   "guess_history": g,
                   "definition": "fp32_over_fp64 = t(pcg64)/t(pmixed); precond_gain = t(mixed)/t(pmixed); "
                                 "net_gain = t(pmixed)/t(" + wl["solver"] + "); fcg_net_gain = t(pmixed)/t(flearned) "
                                 "(flexible CG, net every iteration); guess_gain = t(pmixed, previous-solution "
                                 "guess)/t(pmixed, chronological guess); every arm but the last with the "
                                 "chronological guess of guess_history solutions; same draws and start state"}

    # ---- the fused M^dagger M apply alone, L2 flushed: FP32 against HBM, FP64 against the FP64 rate
    x32 = torch.from_numpy(inputs.complex_gaussian(L, N, 77).astype(np.complex64)).to(dev)
    x64 = torch.from_numpy(inputs.complex_gaussian(L, N, 78)).to(dev)
    us32 = time_apply(hqmc, cfg, theta, x32, flush, hqmc.TIMER_MDAGM32)
    us64 = time_apply(hqmc, cfg, theta, x64, flush, hqmc.TIMER_MDAGM)
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    apply = {"sites": sites,
             "fp32": {"kernel": kernel_name(cfg.launch_shape(hqmc.FP32), "float").replace("CG direction", "apply"),
                      "us": round(us32, 2), "bytes_per_site": 24, "gbs": 24 * sites / us32 / 1e3,
                      "frac_of_measured_hbm": 24 * sites / us32 / 1e3 / hbm},
             "fp64": {"kernel": kernel_name(cfg.launch_shape(hqmc.FP64), "double").replace("CG direction", "apply"),
                      "us": round(us64, 2), "flops_per_site": 126, "tflops": 126 * sites / us64 / 1e6,
                      "frac_of_fp64_rate": 126 * sites / us64 / 1e6 / fp64_tflops if fp64_tflops else None},
             "method": "20 applies, L2 flushed before each (512 MiB write), kernel time from the library's CUDA events"}

    if rank != 0:
        return
    its = [i["cg_iterations"] for i in infos]
    its_per_traj = statistics.mean(its)
    md_avg_ms = md_ms / max(n_md, 1)
    md_med_ms = statistics.median(md_us) / 1e3 if md_us else md_avg_ms
    achieved_tflops = MDAGM_FLOPS_PER_SITE * sites / (md_med_ms * 1e-3) / 1e12
    achieved_gbs = MDAGM_BYTES_PER_SITE[wl["solver"]] * sites / (md_med_ms * 1e-3) / 1e9
    med_up = statistics.median(up_us) if up_us else None
    med_pc = statistics.median(pc_us) if pc_us else None
    shape = cfg.launch_shape(hqmc.FP32 if fp32 else hqmc.FP64)
    kname = kernel_name(shape, "float" if fp32 else "double")
    if fp32:  # the FP32 fused kernel is bounded by HBM bandwidth
        traffic = NCU_TRAFFIC_BYTES.get(wl_name)
        roofline = {"kernel": kname, "bound": "hbm", "achieved": achieved_gbs,
                    "peak": hbm, "unit": "GB/s", "frac": achieved_gbs / hbm, "traffic": traffic,
                    "traffic_note": "DRAM read + write bytes per launch, ncu (profiles/)" if traffic else None,
                    "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                    "bytes_per_site": MDAGM_BYTES_PER_SITE[wl["solver"]], "sites_per_launch": sites,
                    "tflops_algorithmic": achieved_tflops, "launches": n_md,
                    "median_launch_us": 1e3 * md_med_ms, "mean_launch_us_all": 1e3 * md_avg_ms,
                    "launch_time": "median of the per-launch CUDA-event times over one trajectory (launches after "
                                   "a solve converged exit at once; the mean over all launches counts them)",
                    "cg_update_median_us": med_up, "precond_median_us": med_pc,
                    "precond_shape": hqmc.get_precond_shape(cfg, hqmc.FP32)}
    else:
        roofline = {"kernel": kname, "bound": "alu", "achieved": achieved_tflops,
                    "peak": fp64_tflops, "unit": "TFLOP/s", "frac": achieved_tflops / fp64_tflops,
                    "traffic": None,
                    "peak_note": "FP64 FMA rate measured on this GPU by hqmc_probe_fp64_rate",
                    "flops_per_site": MDAGM_FLOPS_PER_SITE, "sites_per_launch": sites,
                    "hbm_gbs_algorithmic": achieved_gbs, "hbm_frac_of_measured": achieved_gbs / hbm,
                    "launches": n_md, "median_launch_us": 1e3 * md_med_ms, "mean_launch_us_all": 1e3 * md_avg_ms,
                    "cg_update_median_us": med_up, "precond_median_us": med_pc}

    # ---- oracle on the host cores: bounded sample --------------------------
    import oracle
    lat = oracle.Lattice(L, N, dtau=wl["dtau"], t=wl["t"], J=wl["J"])
    th_np = start_theta(wl, wl["seed"])
    phi_np = oracle.apply_M(lat, th_np, inputs.complex_gaussian(L, N, wl["seed"] + 1), dagger=True)
    cb = oracle_sample(wl, its_per_traj, th_np, phi_np, max_iters=ORACLE_SAMPLE_ITERS.get(wl_name, 10))

    line = {
        "metric": METRIC, "value": value, "unit": "traj/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if fp32 else "f64", "data": "synthetic",
        "config": config_of(wl_name, wl),
        "e2e": {"value": e2e_value, "unit": "traj/s", "h2d_bytes_per_step": bytes_theta,
                "d2h_bytes_per_step": bytes_theta, "steps": e2e_steps},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "cpu_baseline": {"value": 1.0 / cb["traj_s"], "unit": "traj/s", "cores": cb["cores"], "kind": "oracle",
                         "sample": cb["sample"]},
        "clocks": clk,
        "acceptance": statistics.mean(i["accepted"] for i in infos),
        "acceptance_stderr": (statistics.mean(i["accepted"] for i in infos) *
                              (1 - statistics.mean(i["accepted"] for i in infos)) / len(infos)) ** 0.5,
        "dt": dt,
        "cg_iterations_per_traj": its_per_traj,
        "net_guesses_per_traj": {"tried": statistics.mean(i["net_guesses_tried"] for i in infos),
                                 "kept": statistics.mean(i["net_guesses_used"] for i in infos),
                                 "solves": statistics.mean(i["cg_solves"] for i in infos)},
        "dH": [round(i["dH"], 6) for i in infos],
        "max_true_residual": max(i["max_true_residual"] for i in infos),
        "step_ms": [round(s, 3) for s in step_ms],
        "apply": apply,
    }
    if compare:
        line["vs_plain_fp64"] = compare
    if factors:
        line["factors"] = factors
    if therm:
        line["thermalization"] = therm
    if learned:
        line["learned"] = learned
    print(json.dumps(line), flush=True)
    if net is not None:
        hqmc.set_preconditioner(cfg, None)
        net.close()


def run_batched(args, wl_name, wl, rank, world, local_rank):
    """All chains advance one trajectory per step through hqmc_batch_trajectory; the
    same chains are then run one after another with hqmc_trajectory for comparison."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_16298_gb300 import hqmc, inputs

    torch.cuda.set_device(local_rank)
    lats = BATCH_LATTICES
    seeds = [rank_seed(wl["seed"] + i, rank) for i in range(len(lats))]
    # dt scaled with the volume as in the single-chain workload (|dH| ~ V dt^2)
    dts = [wl["dt"] * ((24 * 24 * 240) / (L * L * N)) ** 0.5 for L, N in lats]
    thetas = [torch.from_numpy(inputs.theta_ordered(L, N, s, tau_walk=0.0)).cuda() for (L, N), s in zip(lats, seeds)]
    stream = torch.cuda.current_stream()
    with hqmc.Batch(lats, autotune=True) as b:
        b.set_solver(wl["solver"])
        shape = b.launch_shape()
        for k in range(args.warmup):
            b.trajectory(thetas, seeds, k, wl["nsteps"], dts, tol=wl["tol"])
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        l0 = b.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = []
        for k in range(args.steps):
            infos.append(b.trajectory(thetas, seeds, args.warmup + k, wl["nsteps"], dts, tol=wl["tol"]))
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        launches = b.launch_count() - l0
    ms = max_over_ranks(ms, world, "cuda")
    value = job_rate(args.steps * len(lats), world, ms / 1e3)
    # the same chains, one trajectory each, run one after another
    seq_ms = 0.0
    for (L, N), s, dt, th in zip(lats, seeds, dts, thetas):
        with hqmc.Config(L, N, variant=1) as cfg:
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            hqmc.trajectory(cfg, th.clone(), seed=s, traj_counter=10 ** 6, nsteps=wl["nsteps"], dt=dt, tol=wl["tol"],
                            solver=wl["solver"])
            z.record(stream)
            torch.cuda.synchronize()
            seq_ms += a.elapsed_time(z)
    if rank != 0:
        return
    flat = [i for step in infos for i in step]
    line = {"metric": METRIC, "value": value, "unit": "traj/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl_name, "chains": len(lats), "lattices": "L in {12,16,20,24} x 8, Ntau = 10 L",
                       "n_leapfrog": wl["nsteps"], "dt": "0.0005 * sqrt(138240 / sites)", "cg_tol": wl["tol"],
                       "solver": wl["solver"] + " (batched: one fused launch + one update launch" +
                                 (" + one preconditioner launch" if wl["solver"] == "pcg64" else "") +
                                 " per CG iteration for all chains)",
                       "batched_tiles": {"cluster": shape["cluster"], "order": ["chain by chain", "largest first",
                                                                                "round robin"][shape["order"]],
                                         "threads": shape["threads"], "autotuned_launch_us": shape["tuned_us"]}},
            "gpu_launches": int(launches),
            "sequential_traj_per_s": len(lats) / (seq_ms / 1e3),
            "batched_over_sequential": value / (len(lats) / (seq_ms / 1e3)),
            "acceptance": sum(i["accepted"] for i in flat) / len(flat),
            "cg_iterations_per_traj": sum(i["cg_iterations"] for i in flat) / len(flat)}
    print(json.dumps(line), flush=True)


def run_estimate(args, wl_name, wl, rank, world, local_rank):
    """A step is one stochastic estimate: nrv vector draws, R = M^dagger xi, nrv solves of
    (M^dagger M) X = R and the mean-diagonal estimate (hqmc_estimate)."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_16298_gb300 import hqmc, inputs

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    L, N, nrv = wl["L"], wl["Ntau"], wl["nrv"]
    cfg = hqmc.Config(L, N, dtau=wl["dtau"], t=wl["t"], J=wl["J"], autotune=True)
    seed = rank_seed(wl["seed"], rank)
    theta = torch.from_numpy(start_theta(wl, seed)).to(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for k in range(args.warmup):
        hqmc.estimate(cfg, theta, nrv, seed=seed, counter=nrv * k, tol=wl["tol"], solver=wl["solver"])
    stream = torch.cuda.current_stream()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    gid = str(local_rank)
    clocks = ClockSampler(gid)
    clocks.start()
    l0 = cfg.launch_count()
    ms, gs, its = [], [], []
    for k in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g, infos, _, _ = hqmc.estimate(cfg, theta, nrv, seed=seed, counter=nrv * (args.warmup + k), tol=wl["tol"],
                                       solver=wl["solver"])
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
        gs.append(g)
        its.append(sum(i["iterations"] for i in infos))
    launches = cfg.launch_count() - l0
    clk = clocks.stop()
    total_ms = sum(ms)
    total_ms = max_over_ranks(total_ms, world, dev)
    value = job_rate(args.steps * nrv, world, total_ms / 1e3)
    if rank != 0:
        return
    cb = oracle_sample(dict(wl, nsteps=-1), statistics.mean(its) / nrv, start_theta(wl, wl["seed"]),
                       inputs.complex_gaussian(L, N, 3), max_iters=ORACLE_SAMPLE_ITERS.get(wl_name, 4))
    cb["sample"] = cb["sample"].replace("and 0 forces per trajectory", "per random vector")
    # the same vectors with the projected initial guesses (hqmc_estimate_projected)
    Gbuf = torch.empty((nrv, N, L, L), dtype=torch.complex128, device=dev)
    hqmc.estimate(cfg, theta, nrv, seed=seed, counter=0, tol=wl["tol"], solver=wl["solver"], projected=True, Gxi=Gbuf)
    pms, pits, pgs = [], [], []
    for k in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g, infos, _, _ = hqmc.estimate(cfg, theta, nrv, seed=seed, counter=nrv * (args.warmup + k), tol=wl["tol"],
                                       solver=wl["solver"], projected=True, Gxi=Gbuf)
        b.record(stream)
        torch.cuda.synchronize()
        pms.append(a.elapsed_time(b))
        pgs.append(g)
        pits.append(sum(i["iterations"] for i in infos))
    projected = {"vectors_per_s": args.steps * nrv / (sum(pms) / 1e3), "iterations_per_vector": statistics.mean(pits) / nrv,
                 "speedup_over_sequential": (sum(ms) / sum(pms)),
                 "estimate_g": [[round(g.real, 6), round(g.imag, 6)] for g in pgs],
                 "method": "each solve starts from the Galerkin projection onto the earlier solutions of the set"}
    # the same vectors with the systems solved together (hqmc_estimate_multi): per CG iteration one
    # tau-walking M^dagger M launch, one update launch and one preconditioner launch for all nrv systems
    hqmc.set_multi_rhs(cfg, nrv)
    shape = hqmc.multi_launch_shape(cfg, nrv)
    for k in range(args.warmup):
        hqmc.estimate(cfg, theta, nrv, seed=seed, counter=nrv * k, tol=wl["tol"], solver=wl["solver"], together=True)
    torch.cuda.synchronize()
    tms, tits, tgs = [], [], []
    l1 = cfg.launch_count()
    for k in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g, infos, _, _ = hqmc.estimate(cfg, theta, nrv, seed=seed, counter=nrv * (args.warmup + k), tol=wl["tol"],
                                       solver=wl["solver"], together=True)
        b.record(stream)
        torch.cuda.synchronize()
        tms.append(a.elapsed_time(b))
        tgs.append(g)
        tits.append(sum(i["iterations"] for i in infos))
    # the multi-system walk launch: CUDA events around every launch of one more estimate (host-driven
    # loop bodies); the median per-launch time (launches after every system converged exit at once)
    hqmc.set_timing(cfg, True)
    hqmc.estimate(cfg, theta, nrv, seed=seed, counter=nrv * (args.warmup + args.steps), tol=wl["tol"],
                  solver=wl["solver"], together=True)
    w_us = hqmc.get_timing_samples(cfg, hqmc.TIMER_MDAGM32)
    u_us = hqmc.get_timing_samples(cfg, hqmc.TIMER_CG_UPDATE)
    p_us = hqmc.get_timing_samples(cfg, hqmc.TIMER_PRECOND)
    hqmc.set_timing(cfg, False)
    sites = L * L * N
    w_med = statistics.median(w_us)
    w_bytes = (32 * nrv + 8) * sites  # per system r/z, p_old, p_new, q (8 B each); theta as float once
    hbm = _peaks().get("hbm_gbs", 6800.0)
    w_gbs = w_bytes / (w_med * 1e-6) / 1e9
    roofline = {"kernel": "hqmc::mdagm_walk_kernel<2, nby, multi> (FP32 M†M, CG direction, %d systems)" % nrv,
                "bound": "hbm", "achieved": w_gbs, "peak": hbm, "unit": "GB/s",
                "frac": w_gbs / hbm if hbm else None, "traffic": None,
                "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                "bytes_per_launch": w_bytes, "bytes_note": "(32 nrv + 8) B per site: per system r or z, p_old, "
                "p_new, q in FP32 complex; theta as float once for all systems",
                "median_launch_us": w_med, "launches": len(w_us),
                "per_system_us": w_med / nrv,
                "cg_update_median_us": statistics.median(u_us) if u_us else None,
                "precond_median_us": statistics.median(p_us) if p_us else None}
    together = {"vectors_per_s": args.steps * nrv / (sum(tms) / 1e3),
                "iterations_per_vector": statistics.mean(tits) / nrv,
                "speedup_over_sequential": sum(ms) / sum(tms), "ms_per_step": sum(tms) / args.steps,
                "gpu_launches": int(cfg.launch_count() - l1),
                "walk_launch": shape,
                "estimate_g": [[round(g.real, 6), round(g.imag, 6)] for g in tgs],
                "step_ms": [round(m, 3) for m in tms],
                "method": "the nrv systems advance together from X = 0: one tau-walking M^dagger M launch "
                          "(CTA b: system b % nrv, slice range b / nrv), one update and one preconditioner "
                          "launch per CG iteration for all systems, one FP64 reliable-update launch per 50"}
    hqmc.set_multi_rhs(cfg, 0)
    line = {"metric": METRIC, "value": value, "unit": "random vectors/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": wl_name, "L": L, "Ntau": N, "sites": L * L * N, "nrv": nrv, "cg_tol": wl["tol"],
                       "solver": SOLVER_TEXT[wl["solver"]], "start": "cold (see hmc workloads)",
                       "l2": "flushed between timed steps"},
            "gpu_launches": int(launches),
            "cpu_baseline": {"value": 1.0 / cb["traj_s"], "unit": "random vectors/s", "cores": cb["cores"],
                             "kind": "oracle", "sample": cb["sample"]},
            "clocks": clk,
            "estimate_g": [[round(g.real, 6), round(g.imag, 6)] for g in gs],
            "exact_re_g": 0.5,
            "iterations_per_vector": statistics.mean(its) / nrv,
            "step_ms": [round(m, 3) for m in ms],
            "projected": projected,
            "together": together,
            "roofline": roofline}
    print(json.dumps(line), flush=True)


def run_profile_case(wl, nrv=None):
    """A short, fixed sequence for ncu captures at the workload's size, with the CG
    loop driven from the host (kernels inside a graph with conditional nodes cannot
    be profiled one by one) and the default launch shapes (an autotuner timed under
    a profiler would not pick the bench's shapes): three fused M^dagger M applies in
    the workload's precision, then one trajectory of 4 leapfrog steps with the
    workload's solver, initial-guess history and first dt (the learned one with a
    freshly initialised net; its cost does not depend on the weights).  For the
    estimate workload: one estimate of nrv vectors (default the workload's) with the
    systems solved together.  Prints no JSON."""
    nrv = nrv or wl.get("nrv")
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_16298_gb300 import hqmc, inputs

    L, N = wl["L"], wl["Ntau"]
    if wl.get("estimate"):  # one estimate with the systems solved together, nrv of them
        with hqmc.Config(L, N, dtau=wl["dtau"], t=wl["t"], J=wl["J"]) as cfg:
            hqmc.set_timing(cfg, True)
            hqmc.set_multi_rhs(cfg, nrv)
            theta = torch.from_numpy(start_theta(wl, wl["seed"])).cuda()
            g, infos, _, _ = hqmc.estimate(cfg, theta, nrv, seed=wl["seed"], tol=wl["tol"], solver=wl["solver"],
                                           together=True)
            torch.cuda.synchronize()
            print("systems:", nrv, "walk launch:", hqmc.multi_launch_shape(cfg, nrv), "iterations per vector:",
                  sum(i["iterations"] for i in infos) / nrv, file=sys.stderr)
        print("profile case done", flush=True)
        return
    with hqmc.Config(L, N, dtau=wl["dtau"], t=wl["t"], J=wl["J"]) as cfg:
        hqmc.set_timing(cfg, True)
        theta = torch.from_numpy(start_theta(wl, wl["seed"])).cuda()
        x = torch.from_numpy(inputs.complex_gaussian(L, N, 2)).cuda()
        xa = x.to(torch.complex64) if wl["solver"] not in ("cg64", "pcg64") else x
        for _ in range(3):
            hqmc.apply_MdagM(cfg, theta, xa)
        net = None
        if wl["solver"] in ("learned", "plearned"):
            net = hqmc.Net(seed=1)
            hqmc.set_preconditioner(cfg, net)
        hqmc.set_guess_history(cfg, wl.get("guess", 0))
        hqmc.trajectory(cfg, theta, seed=wl["seed"], traj_counter=0, nsteps=4, dt=wl["dt"], tol=wl["tol"],
                        solver=wl["solver"])
        torch.cuda.synchronize()
        print("preconditioner shape (FP32):", hqmc.get_precond_shape(cfg, hqmc.FP32), file=sys.stderr)
        if net is not None:
            hqmc.set_preconditioner(cfg, None)
            net.close()
    print("profile case done", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--profile", action="store_true", help="run the short ncu capture case and exit")
    ap.add_argument("--profile-nrv", type=int, default=0,
                    help="estimate workload with --profile: vectors of the estimate (default the workload's)")
    ap.add_argument("--train-triples", type=int, default=0,
                    help="learned workloads: train online on this many sampler triples (none stored) "
                         "instead of epochs over the stored set")
    args = ap.parse_args()
    if args.profile:
        run_profile_case(WORKLOADS[args.workload], args.profile_nrv or None)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    wl = WORKLOADS[args.workload]
    if args.train_triples:
        wl = dict(wl, train_triples=args.train_triples, stream_sources=20)
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if args.impl == "reference":
        run_reference(args, args.workload, wl, rank, world)
    elif wl.get("batched"):
        run_batched(args, args.workload, wl, rank, world, local_rank)
    elif wl.get("estimate"):
        run_estimate(args, args.workload, wl, rank, world, local_rank)
    else:
        run_ours(args, args.workload, wl, rank, world, local_rank)
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
