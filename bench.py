"""Throughput of the GB300 ADER-WENO step: 3-D zone-updates/s.

Workload (default): 3-D Euler, gamma = 1.4, 256^3 periodic unit cube, planar
Sod tube along (1,1,0) (rho 1/0.125, P 1/0.1), third-order nodal ADER-WENO,
HLL flux, CFL 0.4, FP64 -- the 256^3 member of the smooth-advection +
Sod-tube configuration family.  One step = the whole hot path: the CFL dt
reduction (ader_max_dt) then one ADER step with that dt kept on the device
(ader_step_devdt).  The state (671 MB) exceeds L2 (129 MB), so no flush is
needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs an independent problem of the same size (weak
scaling, no collective on the data path).
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

METRIC = "3D zone-updates/s (ADER-WENO step incl. CFL dt reduction)"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    p.add_argument("--n", type=int, default=256)
    p.add_argument("--order", type=int, default=3)
    p.add_argument("--form", default="nodal", choices=["modal", "nodal"])
    p.add_argument("--solver", default="hll", choices=["hll", "linearized"])
    p.add_argument("--fp32", action="store_true")
    p.add_argument("--converged", type=float, default=None,
                   help="converged predictor with this tolerance instead of the fixed M-1 iterations")
    p.add_argument("--learned-guess", action="store_true",
                   help="train the third-order predictor guess first (untimed), then start the converged "
                        "predictor from it (tolerance 1e-6 in FP32, 1e-13 in FP64 unless --converged)")
    p.add_argument("--no-variants", action="store_true", help="skip the per-variant table")
    p.add_argument("--vortex-sizes", default="64,128",
                   help="grid sizes of the 2-D vortex tables (Tables I and II go to 512)")
    p.add_argument("--blast-symmetry", action="store_true",
                   help="also run the 3-D hydrodynamic and MHD blasts to their end times (about ten minutes)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--batch-only", action="store_true",
                   help="only the batched-step comparison (64 and 512 problems), one JSON line of its own")
    p.add_argument("--profile-range", action="store_true",
                   help="with --batch-only: one sequential and one batched step of each set inside "
                        "cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    return p.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(secs, world, device):
    """The slowest rank's timed seconds (every rank returns the same value); world == 1 returns secs."""
    if world <= 1:
        return secs
    import torch
    import torch.distributed as dist
    t = torch.tensor([secs], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank_step, steps, world, secs):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time (weak scaling,
    every rank runs its own problem of the same size)."""
    return units_per_rank_step * steps * world / secs


def cores_used(cpu_s, wall_s):
    """Threads a host run kept busy on average: process CPU time over wall time, at least one."""
    return max(1, int(round(cpu_s / wall_s))) if wall_s > 0 else 1


def host_cores():
    """The host's logical CPU count (the cores the oracle could have used)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- peaks
def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh)
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0, "fallback": True}


def alu_peak_tflops(fp32, sm_mhz):
    """ALU peak from unit counts and clock: 152 SMs; FP64 2 DFMA/clk/SM (the 1.25 TFLOP/s nominal rate
    at 2070 MHz), FP32 128 FFMA/clk/SM; 2 FLOP per FMA."""
    per_clk = 128 * 2 if fp32 else 2 * 2
    return 152 * per_clk * sm_mhz * 1e6 / 1e12


def traffic_per_launch(kernel, order, form, fp32, zones):
    """DRAM bytes per launch of `kernel` from the committed ncu capture, scaled to `zones` (traffic grows
    in proportion to the zones processed); None when the kernel's sources changed since the capture or
    the capture was of another configuration."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic_%s.json" % kernel)
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    if (rec["order"], rec["form"], rec["precision"]) != (order, form, "fp32" if fp32 else "fp64"):
        return None
    h = hashlib.sha256()
    for f in rec["sources"]:
        p = os.path.join(ROOT, f)
        h.update(open(p).read().encode() if os.path.exists(p) else b"")
    if h.hexdigest() != rec["sources_sha256"]:
        return None
    return rec["bytes_per_zone"] * zones


UPDATE_FLOPS = 3 * 5 * 3 + 5 * 2      # Eq. 6 from stored fluxes: per direction and variable a subtract, a
                                      # multiply and a subtract, then base + c acc (the counter's "acc" term)


def flops_per_zone(order, form, solver, fp32, tiled=True):
    """Exact FLOPs per zone of each kernel (op-counting instantiation of the kernels' per-zone code).

    Tiled layout (Euler, orders 2-3): the predictor kernel also solves each face once, so it carries the
    face solves and the update kernel only Eq. 6 from the stored fluxes."""
    path = os.path.join(ROOT, "paper_1006_2146_gb300", "flops.json")
    if not os.path.exists(path):
        return {}
    with open(path) as fh:
        f = json.load(fh)["order%d" % order]
    if tiled and order <= 3:
        solves = f["riemann_update_" + solver] - UPDATE_FLOPS
        return {"weno_reconstruction": f["weno_reconstruction"],
                "predictor_faces": f["predictor_faces_" + form] + solves,
                "riemann_update": UPDATE_FLOPS}
    return {"weno_reconstruction": f["weno_reconstruction"],
            "predictor_faces": f["predictor_faces_" + form],
            "riemann_update": f["riemann_update_" + ("fused_" if fp32 else "") + solver]}


# ----------------------------------------------------------------------------- GPU arm
def rel_l1_dev(got, want):
    """max over variables of sum|got - want| / max(sum|want_v|, sum|rho|) (the parity measure), on the device."""
    num = (got - want).abs().reshape(want.shape[0], -1).sum(dim=1)
    den = want.abs().reshape(want.shape[0], -1).sum(dim=1)
    den = den.clamp(min=float(den[0]))
    return float((num / den).max())


def mhd_variants(ader, torch, stream, n=128, steps=3, warmup=1):
    """Ideal MHD, Orszag-Tang-type vortex extruded in z (n^3, gamma 5/3, third order, modal): zone-updates/s
    per configuration, and the relative max |div B| after the timed steps (ader_diagnostics)."""
    from paper_1006_2146_gb300 import _lib, inputs
    out = {}
    try:
        U0, B0 = inputs.orszag_tang(n)
    except Exception as exc:
        return {"mhd_inputs": {"error": str(exc)[:200]}}
    U0 = torch.from_numpy(U0).to("cuda")
    B0 = torch.from_numpy(B0).to("cuda")
    zones = n ** 3
    for name, fp32, solver in (("mhd_ot_fp32_linearized_o3", True, "linearized"),
                               ("mhd_ot_fp32_hll_o3", True, "hll"),
                               ("mhd_ot_fp32_hll_o3_emf_transonic", True, "hll"),
                               ("mhd_ot_fp64_linearized_o3", False, "linearized"),
                               ("mhd_ot_fp32_ssprk3_linearized_o3", True, "linearized")):
        rk = "ssprk" in name
        h = None
        try:
            flags = _lib.ADER_MHD | (_lib.ADER_FP32_BULK if fp32 else 0) | \
                (_lib.ADER_EMF_TRANSONIC if name.endswith("emf_transonic") else 0)
            h = _lib.ader_create(n, n, n, 1.0 / n, 1.0 / n, 1.0 / n, 3, 5.0 / 3.0,
                                 _lib.ADER_LINEARIZED if solver == "linearized" else _lib.ADER_HLL, flags)
            d, b = U0.clone(), B0.clone()
            dt = torch.zeros(1, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()                    # the copies (current stream) before `stream` reads them
            _lib.ader_max_dt(h, d, b, 0.4, dt, stream)
            torch.cuda.synchronize()
            dt_rk = 0.5 * float(dt.item())            # SSP-RK3 at half the ADER step (host dt: its stages)
            with torch.cuda.stream(stream):
                for _ in range(warmup):
                    if rk:
                        _lib.ader_rk_step(h, d, b, dt_rk, stream)
                    else:
                        _lib.ader_max_dt(h, d, b, 0.4, dt, stream)
                        _lib.ader_step_devdt(h, d, b, dt, stream)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(steps):
                    if rk:
                        _lib.ader_rk_step(h, d, b, dt_rk, stream)
                    else:
                        _lib.ader_max_dt(h, d, b, 0.4, dt, stream)
                        _lib.ader_step_devdt(h, d, b, dt, stream)
                e1.record(stream)
            torch.cuda.synchronize()
            secs = e0.elapsed_time(e1) / 1e3
            diag = torch.zeros(9, dtype=torch.float64, device="cuda")
            _lib.ader_diagnostics(h, d, b, diag, stream)
            st = _lib.ader_sync_status(h, stream)
            out[name] = {"zone_updates_per_s": zones * steps / secs, "ms_per_step": secs / steps * 1e3,
                         "grid": n, "status": st, "div_b_rel_after": float(diag[8].item())}
        except Exception as exc:
            out[name] = {"error": str(exc)[:200]}
        finally:
            if h is not None:
                _lib.ader_destroy(h)
    return out


def mhd_learned_evaluation(ader, torch, stream, n=128, steps=3, train_n=96):
    """The learned guess for ideal MHD on the unseen n^3 Orszag-Tang-type vortex (third order, modal,
    linearized solver).  The MHD network is trained first (outside every timed region) on predictor samples
    of the seeded magnetised training states at train_n^3.  Each run starts from the same state, takes one
    warm-up step, then `steps` timed steps of one fixed dt; it reports the mean predictor iterations and,
    for FP32, the error against the FP64 converged predictor (the reference for the guess's error)."""
    from paper_1006_2146_gb300 import _lib, inputs, learned
    out = {}
    try:
        t0 = time.perf_counter()
        X, Y = learned.make_samples(learned.training_states(train_n, mhd=True), train_n, mhd=True)
        t1 = time.perf_counter()
        P, losses = learned.train(X, Y, mhd=True)
        torch.cuda.synchronize()
        out["training"] = {"samples": int(X.shape[0]), "epochs": len(losses), "first_epoch_loss": losses[0],
                           "final_loss": losses[-1], "sample_s": t1 - t0, "train_s": time.perf_counter() - t1}
        del X, Y
        Uh, Bh = inputs.orszag_tang(n)
        U0 = torch.from_numpy(Uh).to("cuda")
        B0 = torch.from_numpy(Bh).to("cuda")
    except Exception as exc:
        out["error"] = str(exc)[:200]
        return out
    zones = n ** 3

    def run(fp32, tol, guess):
        flags = _lib.ADER_MHD | (_lib.ADER_FP32_BULK if fp32 else 0)
        h = _lib.ader_create(n, n, n, 1.0 / n, 1.0 / n, 1.0 / n, 3, 5.0 / 3.0, _lib.ADER_LINEARIZED, flags)
        try:
            dtv = torch.zeros(1, dtype=torch.float64, device="cuda")
            _lib.ader_max_dt(h, U0, B0, 0.4, dtv, stream)
            torch.cuda.synchronize()
            dt = float(dtv.item())
            _lib.ader_set_predictor(h, tol, 50)
            if guess is not None:
                _lib.ader_set_guess(h, guess)
            d, b = U0.clone(), B0.clone()
            torch.cuda.synchronize()                    # the copies (current stream) before `stream` reads them
            _lib.ader_step(h, d, b, dt, stream)                 # warm-up step, counts discarded
            torch.cuda.synchronize()
            _lib.ader_predictor_stats(h, stream)
            d, b = U0.clone(), B0.clone()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                for _ in range(steps):
                    _lib.ader_step(h, d, b, dt, stream)
                e1.record(stream)
            torch.cuda.synchronize()
            secs = e0.elapsed_time(e1) / 1e3
            tot, mx, capped = _lib.ader_predictor_stats(h, stream)
            st = _lib.ader_sync_status(h, stream)
        finally:
            _lib.ader_destroy(h)
        return d, b, {"zone_updates_per_s": zones * steps / secs, "ms_per_step": secs / steps * 1e3,
                      "mean_predictor_iterations": tot / (steps * zones), "max_predictor_iterations": mx,
                      "capped": capped, "status": st, "tol": tol}

    try:
        ref_d, ref_b, rec = run(False, 1e-13, None)
        out["fp64_converged"] = rec
        for name, fp32, tol, guess in (("fp64_converged_learned_guess", False, 1e-13, P),
                                       ("fp32_converged", True, 1e-6, None),
                                       ("fp32_converged_learned_guess", True, 1e-6, P)):
            d, b, rec = run(fp32, tol, guess)
            rec["rel_l1_vs_fp64_converged_%dsteps" % steps] = rel_l1_dev(d, ref_d)
            rec["face_b_rel_l1_vs_fp64_converged"] = float((b - ref_b).abs().sum() / ref_b.abs().sum())
            out[name] = rec
    except Exception as exc:
        out["error"] = str(exc)[:200]
    try:
        out["accuracy_bound"] = guess_accuracy_bound(ader, torch, P, U0, B0, form="modal", solver="linearized",
                                                     gamma=5.0 / 3.0, stream=stream)
    except Exception as exc:
        out["accuracy_bound"] = {"error": str(exc)[:200]}
    return out


def convergence_variant(ader, torch, sizes=(32, 64, 128), T=0.05):
    """L1 error of rho on the config-1 density wave (FP64, nodal, HLL, CFL 0.4) at each size and order,
    and the rates between sizes: the 3-D analogue of the paper's Table IV (whose own setup differs)."""
    from paper_1006_2146_gb300 import inputs
    import numpy as np
    out = {}
    for order in (2, 3, 4):
        errs = []
        for n in sizes:
            s = ader.Solver((n, n, n), order=order, form="nodal")
            d = torch.from_numpy(inputs.density_wave(n)).to("cuda")
            dtv = torch.zeros(1, dtype=torch.float64, device="cuda")
            t = 0.0
            while t < T - 1e-14:
                s.max_dt(d, 0.4, dtv)
                dt = min(float(dtv.item()), T - t)
                s.step(d, dt)
                t += dt
            st = s.status()
            s.close()
            exact = torch.from_numpy(inputs.density_wave(n, t=T)[0]).to("cuda")
            errs.append(float((d[0] - exact).abs().mean()) if st == 0 else None)
        rates = [float(np.log2(errs[i] / errs[i + 1])) if errs[i] and errs[i + 1] else None
                 for i in range(len(sizes) - 1)]
        out["order%d" % order] = {"sizes": list(sizes), "l1_rho": errs, "rates": rates}
    out["paper_table_iv_rates_64_to_96"] = {"order2": 2.31, "order3": 2.97, "order4": 4.01}
    return out


def vortex_tables(ader, torch, sizes=(64, 128, 256)):
    """The paper's Tables I and II on this path: the 2-D isentropic (Sec. VI.1) and magnetised (Sec. VI.2)
    vortices as one-zone z-slabs, FP64, modal, HLL, CFL 0.45, run for one period of the mean flow (t = 10 on
    [-5, 5]^2; t = 20 on [-10, 10]^2 at fourth order).  Per zone L1 / Linf error of rho (Table I) and of the
    x-face field (Table II), the rates, and the paper's printed L1 errors beside them."""
    from paper_1006_2146_gb300 import inputs, run
    import numpy as np
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden", "vortex_tables.json")) as fh:
        paper = json.load(fh)
    idx = [paper["sizes"].index(n) for n in sizes]
    out = {}
    for table, kind in (("table_i", "hydro"), ("table_ii", "mhd")):
        res = {}
        for order in (2, 3, 4):
            L = 20.0 if order == 4 else 10.0
            l1, linf, secs = [], [], 0.0
            for n in sizes:
                if kind == "hydro":
                    U, B, G = inputs.isentropic_vortex(n, L=L), None, 1.4
                else:
                    (U, B), G = inputs.magnetized_vortex(n, L=L), 5.0 / 3.0
                s = ader.Solver((1, n, n), order=order, form="modal", solver="hll", gamma=G,
                                lengths=inputs.slab_lengths(L), mhd=(B is not None))
                dU = torch.from_numpy(U).to("cuda")
                dB = None if B is None else torch.from_numpy(B).to("cuda")
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                run.advance(s, dU, L, cfl=0.45, Bface=dB)
                torch.cuda.synchronize()
                secs += time.perf_counter() - t0
                s.close()
                err = (dU[0].cpu().numpy() - U[0]) if B is None else (dB[0].cpu().numpy() - B[0])
                l1.append(float(np.abs(err).mean()))
                linf.append(float(np.abs(err).max()))
            res["order%d" % order] = {
                "sizes": list(sizes), "l1": l1, "linf": linf,
                "l1_rates": [float(np.log2(l1[i] / l1[i + 1])) for i in range(len(sizes) - 1)],
                "paper_l1": [paper[table]["order%d" % order]["l1"][i] for i in idx],
                "seconds": secs}
        out[table] = res
    return out


# Nodal asymmetry of the final velocities printed by the paper (fractions): Sec. VIII.3 (hydrodynamic blast,
# 96^3, t = 0.1) and Sec. IX.4 (MHD blast, 97^3, t = 0.014); the modal schemes are symmetric to round-off.
PAPER_NODAL_ASYMMETRY = {"hydro_blast_96": {"order2": 4e-4, "order3": 2e-6, "order4": 7e-5},
                         "mhd_blast_97": {"order2": 2.1e-5, "order3": 1.4e-3, "order4": 7.1e-5}}


def velocity_asymmetry(torch, U):
    """Departures from the point symmetry through the domain centre that a centred blast keeps (v odd;
    rho, P and B even): (pointwise, peak).  pointwise = max over zones and components of |v(x) + v(-x)|
    / max |v|; peak = max over directions d of |max v_d - max(-v_d)| / max |v_d|, the difference between
    the largest velocities in opposite directions."""
    v = U[1:4] / U[0]
    pointwise = float((v + torch.flip(v, dims=(1, 2, 3))).abs().max() / v.abs().max())
    peak = max(float((v[d].max() - (-v[d]).max()).abs() / v[d].abs().max()) for d in range(3))
    return pointwise, peak


def blast_symmetry(ader, torch, orders=(2, 3, 4), forms=("modal", "nodal"),
                   cases=(("hydro_blast_96", "hll"), ("mhd_blast_97", "hll"), ("mhd_blast_97", "linearized"),
                          ("mhd_blast_97", "hll_emf_transonic"), ("hydro_blast_96", "hll_positivity"),
                          ("mhd_blast_97", "hll_positivity"), ("mhd_blast_97", "linearized_positivity"))):
    """The paper's 3-D blasts run to their end times at CFL 0.3 (FP64): the velocity asymmetry of each
    order and form beside the printed nodal figures, the step count and wall time, or the error status
    of a run that does not finish (the robustness half of the test)."""
    from paper_1006_2146_gb300 import _lib, inputs, run
    out = {}
    for name, solver in cases:
        mhd = name.startswith("mhd")
        n, T = (97, 0.014) if mhd else (96, 0.1)
        U, B = inputs.mhd_blast(n) if mhd else (inputs.blast(n), None)
        res = {"n": n, "t_end": T, "solver": solver, "paper_nodal_asymmetry": PAPER_NODAL_ASYMMETRY[name]}
        for order in orders:
            for form in forms:
                s = ader.Solver((n, n, n), order=order, form=form, solver=solver.split("_")[0], gamma=1.4,
                                mhd=mhd, emf_transonic=solver.endswith("emf_transonic"),
                                positivity=solver.endswith("positivity"))
                dU = torch.from_numpy(U).to("cuda")
                dB = None if B is None else torch.from_numpy(B).to("cuda")
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                try:
                    t, steps = run.advance(s, dU, T, cfl=0.3, Bface=dB, max_steps=20000)
                    torch.cuda.synchronize()
                    pw, pk = velocity_asymmetry(torch, dU)
                    rec = {"asymmetry_pointwise": pw, "asymmetry_peak": pk, "steps": steps, "t": t,
                           "seconds": time.perf_counter() - t0, "rho_min": float(dU[0].min())}
                except _lib.AderError as exc:
                    rec = {"error": str(exc)[:200]}
                s.close()
                res["%s_order%d" % (form, order)] = rec
        out["%s_%s" % (name, solver)] = res
    return out


def dense_output_variant(ader, torch, stream, n, U0, reps=5):
    """Dense output (Sec. VII) on the headline workload: the step with and without keeping the space-time
    modes, and the evaluation kernel at tau = 1/2 with its HBM rate (it reads L x 5 and writes LS x 5 FP64
    values per zone: 1,000 B at third order)."""
    L, LS = 15, 10
    s = ader.Solver((n, n, n), order=3, form="nodal")
    d = U0.clone()
    out = torch.empty((LS, 5, n, n, n), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    dtv = torch.zeros(1, dtype=torch.float64, device="cuda")
    res = {}
    with torch.cuda.stream(stream):
        s.max_dt(d, 0.4, dtv, stream)
        dt = 0.5 * float(dtv.item())

        def timed(fn):
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1) / reps
        res["step_ms_plain"] = timed(lambda: s.step(d, dt, stream))
        s.set_dense_output(True)
        res["step_ms_keeping_modes"] = timed(lambda: s.step(d, dt, stream))
        ms = timed(lambda: s.dense_output(0.5, out, stream))
    s.close()
    zones = n ** 3
    gbs = (L + LS) * 5 * 8 * zones / (ms * 1e-3) / 1e9
    res.update({"eval_ms": ms, "eval_bytes_per_zone": (L + LS) * 5 * 8, "eval_gbs": gbs,
                "eval_frac_of_measured_hbm": gbs / peaks().get("hbm_gbs", 6800.0)})
    return res


def batched_variant(ader, torch, stream, steps=3, warmup=1, count=64, sizes=(32, 48, 64, 80, 96, 112, 128),
                    profile_range=False):
    """`count` seeded independent problems of uneven cubic sizes (Euler and MHD, orders 2-4, FP32 bulk):
    one tuned batch replayed from a captured graph vs one context per problem launched in sequence.
    Each step includes every problem's CFL dt.  profile_range: after the timing, one more step of each
    inside cudaProfilerStart/Stop."""
    from paper_1006_2146_gb300 import _lib, inputs
    trim_local_memory(_lib)                           # the layout the batch's own kernels need (run_config)
    t0 = time.perf_counter()
    probs = inputs.batch_problems(count, seed=1006, sizes=sizes)
    gen_s = time.perf_counter() - t0
    zones = sum(p["U"][0].size for p in probs)
    Us = [torch.from_numpy(p["U"]).to("cuda") for p in probs]
    Bs = [torch.from_numpy(p["B"]).to("cuda") if p["mhd"] else None for p in probs]
    out = {"problems": len(probs), "zones": int(zones), "input_generation_s": gen_s,
           "sizes": sorted(set(p["shape"][0] for p in probs))}

    def flags_of(p):
        return (_lib.ADER_FP32_BULK | (_lib.ADER_NODAL if p["form"] == "nodal" else 0) |
                (_lib.ADER_MHD if p["mhd"] else 0))

    def solver_of(p):
        return _lib.ADER_LINEARIZED if p["solver"] == "linearized" else _lib.ADER_HLL

    # sequential: one context per problem
    hs = []
    try:
        dts = torch.zeros(len(probs), dtype=torch.float64, device="cuda")
        for p in probs:
            n = p["shape"][0]
            hs.append(_lib.ader_create(n, n, n, 1.0 / n, 1.0 / n, 1.0 / n, p["order"], p["gamma"], solver_of(p),
                                       flags_of(p)))
        d = [u.clone() for u in Us]
        db = [None if x is None else x.clone() for x in Bs]
        torch.cuda.synchronize()                        # the copies (current stream) before `stream` reads them

        def seq_step():
            for k, h in enumerate(hs):
                _lib.ader_max_dt(h, d[k], db[k], 0.4, dts[k:k + 1], stream)
                _lib.ader_step_devdt(h, d[k], db[k], dts[k:k + 1], stream)

        with torch.cuda.stream(stream):
            for _ in range(warmup):
                seq_step()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                seq_step()
            e1.record(stream)
        torch.cuda.synchronize()
        seq_s = e0.elapsed_time(e1) / 1e3
        if profile_range:
            torch.cuda.cudart().cudaProfilerStart()
            with torch.cuda.stream(stream):
                seq_step()
            torch.cuda.synchronize()
            torch.cuda.cudart().cudaProfilerStop()
        bad = [k for k, h in enumerate(hs) if _lib.ader_sync_status(h, stream) != 0]
        out["sequential"] = {"zone_updates_per_s": zones * steps / seq_s, "ms_per_step": seq_s / steps * 1e3,
                             "launches_per_step": sum(_lib.ader_launches_per_step(h) + 1 for h in hs),
                             "problems_with_errors": bad}
        del d, db
    except Exception as exc:
        out["sequential"] = {"error": str(exc)[:200]}
    finally:
        for h in hs:
            _lib.ader_destroy(h)
    # batched: tune, then the captured step
    b = None
    try:
        n3 = [p["shape"][0] for p in probs]
        b = _lib.ader_batch_create([(n, n, n, 1.0 / n, 1.0 / n, 1.0 / n) for n in n3], [p["order"] for p in probs],
                                   [p["gamma"] for p in probs], [solver_of(p) for p in probs],
                                   [flags_of(p) for p in probs])
        d = [u.clone() for u in Us]
        db = [None if x is None else x.clone() for x in Bs]
        dtb = torch.zeros(len(probs), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()                        # the copies (current stream) before `stream` reads them
        t0 = time.perf_counter()
        _lib.ader_batch_tune(b, d, db, stream)
        tune_s = time.perf_counter() - t0
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                _lib.ader_batch_advance(b, d, db, 0.4, dtb, stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                _lib.ader_batch_advance(b, d, db, 0.4, dtb, stream)
            e1.record(stream)
        torch.cuda.synchronize()
        bs = e0.elapsed_time(e1) / 1e3
        if profile_range:
            torch.cuda.cudart().cudaProfilerStart()
            with torch.cuda.stream(stream):
                _lib.ader_batch_advance(b, d, db, 0.4, dtb, stream)
            torch.cuda.synchronize()
            torch.cuda.cudart().cudaProfilerStop()
        rc, codes = _lib.ader_batch_status(b, len(probs), stream)
        out["batched"] = {"zone_updates_per_s": zones * steps / bs, "ms_per_step": bs / steps * 1e3,
                          "graph_launches_per_step": 1, "groups": _lib.ader_batch_groups(b), "tune_s": tune_s,
                          "status": rc, "tuned_shapes": _lib.ader_batch_tuning(b)}
        if "zone_updates_per_s" in out.get("sequential", {}):
            out["speedup_vs_sequential"] = out["batched"]["zone_updates_per_s"] / out["sequential"]["zone_updates_per_s"]
    except Exception as exc:
        out["batched"] = {"error": str(exc)[:200]}
    finally:
        if b is not None:
            _lib.ader_batch_destroy(b)
    return out


def guess_accuracy_bound(ader, torch, P, U0, B0=None, form="modal", solver="hll", gamma=1.4, stream=None):
    """What a guess must reach to save an iteration, measured on one step of a state (FP64, third order).

    The predictor's polynomial at the end of the step minus at its start (dense output at tau = 1 and 0) is
    its evolutionary part: u11 + u12, u13, u14, u15 per variable.  Its relative L2 error against the
    converged predictor (tol 1e-13) is taken for the learned guess (ader_guess_eval) and for k = 1, 2, 3
    Picard iterations from zero (the converged mode capped at k).  Starting from the guess saves the first
    k iterations only where the guess is at least as accurate as k iterations from zero: e_guess < e_1 is
    the bound the network must meet to pay at all."""
    from paper_1006_2146_gb300 import _lib
    mhd = B0 is not None
    nz, ny, nx = U0.shape[1:]
    nv = 8 if mhd else 5
    zones = nx * ny * nz
    flags = (_lib.ADER_MHD if mhd else 0) | (_lib.ADER_NODAL if form == "nodal" else 0)
    sol = _lib.ADER_HLL if solver == "hll" else _lib.ADER_LINEARIZED

    def make():
        return _lib.ader_create(nx, ny, nz, 1.0 / nx, 1.0 / ny, 1.0 / nz, 3, gamma, sol, flags)

    h = make()
    dtv = torch.zeros(1, dtype=torch.float64, device="cuda")
    _lib.ader_max_dt(h, U0, B0, 0.4, dtv, stream)
    torch.cuda.synchronize()
    dt = float(dtv.item())
    _lib.ader_destroy(h)

    def increment(max_iter):
        h = make()
        try:
            _lib.ader_set_predictor(h, 1e-13, max_iter)
            _lib.ader_set_dense_output(h, True)
            d = U0.clone()
            b = B0.clone() if mhd else None
            torch.cuda.synchronize()
            _lib.ader_step(h, d, b, dt, stream)
            w0 = torch.empty((10, nv, zones), dtype=torch.float64, device="cuda")
            w1 = torch.empty_like(w0)
            _lib.ader_dense_output(h, 0.0, w0, stream)
            _lib.ader_dense_output(h, 1.0, w1, stream)
            torch.cuda.synchronize()
            _lib.ader_sync_status(h, stream)            # a capped run reports ADER_ERR_NOT_CONVERGED: expected
        finally:
            _lib.ader_destroy(h)
        return (w1 - w0)[:4]                            # modes 1-4 carry the evolutionary part at tau = 1

    ref = increment(50)
    h = make()
    try:
        _lib.ader_set_guess(h, P)
        G = torch.zeros((25 if not mhd else 40, zones), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        _lib.ader_guess_eval(h, U0, B0, dt, G, stream)
        torch.cuda.synchronize()
        st = _lib.ader_sync_status(h, stream)
    finally:
        _lib.ader_destroy(h)
    Gd = G.double().reshape(5, nv, zones)               # u11..u15 of each variable
    guess = torch.stack([Gd[0] + Gd[1], Gd[2], Gd[3], Gd[4]])
    norm = float(ref.norm())

    def err(x):
        return float((x - ref).norm()) / norm if norm > 0 else 0.0

    out = {"e_guess": err(guess), "guess_status": st, "dt": dt}
    for k in (1, 2, 3):
        out["e_%d_iterations_from_zero" % k] = err(increment(k))
    out["guess_saves_an_iteration"] = out["e_guess"] < out["e_1_iterations_from_zero"]
    return out


def blast_evaluation(ader, torch, P, stream, n=256, steps=3):
    """The learned guess on the 256^3 hydrodynamic blast (Sec. VIII.3 set-up: rho = 1, P 1000 inside r < 0.1,
    0.1 outside): FP32 converged predictor (tol 1e-6) from zero and from the guess, timed, with the mean
    iteration count and the error after `steps` steps of one fixed dt against the FP64 converged predictor."""
    from paper_1006_2146_gb300 import inputs
    out = {}
    try:
        U0 = torch.from_numpy(inputs.blast(n, sub=2)).to("cuda")
        s = ader.Solver((n, n, n), order=3, form="nodal")
        dtv = torch.zeros(1, dtype=torch.float64, device="cuda")
        s.max_dt(U0, 0.4, dtv)
        s.close()
        dt = float(dtv.item())

        def run(fp32, tol, guess, timed):
            s = ader.Solver((n, n, n), order=3, form="nodal", fp32=fp32)
            s.set_predictor(tol, 50)
            if guess is not None:
                s.set_guess(guess)
            d = U0.clone()
            torch.cuda.synchronize()                    # the copy (current stream) before `stream` reads it
            s.step(d, dt, stream)                       # warm-up step, discarded counts
            torch.cuda.synchronize()
            s.predictor_stats(stream)
            d = U0.clone()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                for _ in range(steps):
                    s.step(d, dt, stream)
                e1.record(stream)
            torch.cuda.synchronize()
            tot, mx, capped = s.predictor_stats(stream)
            st = s.status(stream)
            s.close()
            rec = {"ms_per_step": e0.elapsed_time(e1) / steps, "zone_updates_per_s": n ** 3 * steps /
                   (e0.elapsed_time(e1) / 1e3), "mean_predictor_iterations": tot / (steps * n ** 3),
                   "max_predictor_iterations": mx, "capped": capped, "status": st}
            return d, rec

        ref, rec = run(False, 1e-13, None, True)
        out["fp64_converged"] = rec
        for name, guess in (("fp32_converged", None), ("fp32_converged_learned_guess", P)):
            d, rec = run(True, 1e-6, guess, True)
            rec["rel_l1_vs_fp64_converged_%dsteps" % steps] = rel_l1_dev(d, ref)
            out[name] = rec
    except Exception as exc:
        out["error"] = str(exc)[:200]
    return out


def learned_variants(ader, torch, n, U0, stream, steps=3):
    """Converged predictor from zero and from the learned guess (third order, nodal, HLL).

    The guess is trained first (outside every timed region) on predictor samples of the seeded training
    states at 128^3 (about 10^7 samples).  Each variant is timed like the headline; its state after `steps`
    steps of one fixed dt is compared with the FP64 converged predictor's (the reference for the guess's error)
    and with the FP64 fixed-iteration method.
    """
    from paper_1006_2146_gb300 import learned
    out = {}
    try:
        t0 = time.perf_counter()
        X, Y = learned.make_samples(learned.training_states(128), 128)
        t1 = time.perf_counter()
        P, losses = learned.train(X, Y)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        out["learned_guess_training"] = {"samples": int(X.shape[0]), "epochs": len(losses), "final_loss": losses[-1],
                                         "first_epoch_loss": losses[0], "sample_s": t1 - t0, "train_s": t2 - t1}
        del X, Y
    except Exception as exc:
        return {"learned_guess_training": {"error": str(exc)[:200]}}
    zones = n ** 3
    cases = [("fp64_converged_nodal_o3", False, 1e-13, None), ("fp32_converged_nodal_o3", True, 1e-6, None),
             ("fp32_learned_guess_nodal_o3", True, 1e-6, P), ("fp64_learned_guess_nodal_o3", False, 1e-13, P)]
    dtv = torch.zeros(1, dtype=torch.float64, device="cuda")
    sref = ader.Solver((n, n, n), order=3, form="nodal")
    sref.max_dt(U0, 0.4, dtv)
    sref.close()
    dt_fixed = float(dtv.item())

    def fixed_run(fp32, tol, guess):
        s = ader.Solver((n, n, n), order=3, form="nodal", fp32=fp32)
        if tol is not None:
            s.set_predictor(tol, 50)
        if guess is not None:
            s.set_guess(guess)
        d = U0.clone()
        for _ in range(steps):
            s.step(d, dt_fixed)
        st = s.status()
        s.close()
        if st != 0:
            raise RuntimeError("device status %d" % st)
        return d

    try:
        ref = fixed_run(False, 1e-13, None)
        plain = fixed_run(False, None, None)
        out["fp64_plain_vs_converged_rel_l1"] = rel_l1_dev(plain, ref)
        del plain
    except Exception as exc:
        ref = None
        out["fp64_converged_reference"] = {"error": str(exc)[:200]}
    out["learned_guess_on_blast_256"] = blast_evaluation(ader, torch, P, stream)
    try:
        from paper_1006_2146_gb300 import inputs
        Ub = torch.from_numpy(inputs.blast(128, sub=2)).to("cuda")
        out["learned_guess_accuracy_bound_blast_128"] = guess_accuracy_bound(ader, torch, P, Ub, form="nodal",
                                                                             stream=stream)
        Ur = torch.from_numpy(inputs.random_smooth((64, 64, 64), seed=1006, amp=0.3)).to("cuda")
        out["learned_guess_accuracy_bound_random_64"] = guess_accuracy_bound(ader, torch, P, Ur, form="nodal",
                                                                             stream=stream)
        del Ub, Ur
    except Exception as exc:
        out["learned_guess_accuracy_bound_blast_128"] = {"error": str(exc)[:200]}
    for name, fp32, tol, guess in cases:
        try:
            vsecs, vprof, vs_, _, _ = run_config(ader, torch, n, 3, "nodal", "hll", fp32, 3, 1, stream, profile=True,
                                                 state=U0, tol=tol, guess=guess)
            tot, mx, capped = vs_.predictor_stats(stream)
            vs_.close()
            rec = {"zone_updates_per_s": zones * 3 / vsecs, "ms_per_step": vsecs / 3 * 1e3,
                   "kernel_ms": {k: round(v[1] / v[0], 3) for k, v in vprof.items()},
                   "mean_predictor_iterations": tot / (3.0 * zones), "max_predictor_iterations": mx,
                   "tol": tol}
            if ref is not None:
                d = fixed_run(fp32, tol, guess)
                rec["rel_l1_vs_fp64_converged_%dsteps" % steps] = rel_l1_dev(d, ref)
                del d
            out[name] = rec
        except Exception as exc:
            out[name] = {"error": str(exc)[:200]}
    return out



def trim_local_memory(lib):
    """ader_trim_local_memory, best effort: housekeeping between configurations, never a reason to fail."""
    try:
        lib.ader_trim_local_memory()
    except Exception as exc:                           # noqa: BLE001 - reported, not fatal
        print("note: local memory not trimmed (%s)" % exc, file=sys.stderr)


def run_config(ader, torch, n, order, form, solver, fp32, steps, warmup, stream, profile=False, state=None,
               tol=None, guess=None, source=None, tiled=True):
    """Times `steps` steps of max_dt + step_devdt; returns (seconds, profile dict, solver, device state).

    tol: converged predictor (iterate to tol, at most 50 times); guess: learned-guess parameters (device);
    source: (kind, params) of Solver.set_source; tiled: the Euler launch layout (ader_set_tiled).
    """
    from paper_1006_2146_gb300 import inputs
    # each configuration in the local-memory layout its own kernels need, as when run alone (a fourth-order
    # FP64 run before it would otherwise leave every later kernel a 5 KB-per-thread stack)
    trim_local_memory(ader)
    s = ader.Solver((n, n, n), order=order, form=form, solver=solver, fp32=fp32)
    s.set_tiled(tiled)
    if source is not None:
        s.set_source(*source)
    if tol is not None:
        s.set_predictor(tol, 50)
    if guess is not None:
        s.set_guess(guess)
    if state is None:
        state = torch.from_numpy(inputs.sod_planar(n)).to("cuda")
    d = state.clone()
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()                            # the copy (current stream) before `stream` reads it
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            s.max_dt(d, 0.4, dt, stream)
            s.step_devdt(d, dt, stream)
    torch.cuda.synchronize()
    if tol is not None:
        s.predictor_stats(stream)          # clears the counts of the warm-up steps
    if profile:
        ader.ader_profile(s.h, True)
        ader.ader_profile_reset(s.h)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(steps):
            s.max_dt(d, 0.4, dt, stream)
            s.step_devdt(d, dt, stream)
        e1.record(stream)
    torch.cuda.synchronize()
    prof = ader.ader_profile_read(s.h) if profile else None
    status = s.status(stream)
    launches = ader.ader_launches_per_step(s.h) + 1
    if status != 0:
        raise RuntimeError("device status %d after the timed steps: %s" % (status, ader.ader_last_error(s.h)))
    return e0.elapsed_time(e1) / 1e3, prof, s, d, launches


def gpu_arm(args):
    import numpy as np
    import torch

    import paper_1006_2146_gb300 as ader
    from paper_1006_2146_gb300 import inputs

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    ader.load()
    stream = torch.cuda.Stream()
    if args.batch_only:
        res = {"batched_64_problems_fp32": batched_variant(ader, torch, stream, profile_range=args.profile_range),
               "batched_512_small_problems_fp32": batched_variant(ader, torch, stream, count=512, sizes=(16, 24, 32),
                                                                  profile_range=args.profile_range)}
        for r in res.values():
            r.get("batched", {}).pop("tuned_shapes", None)
        if rank == 0:
            print(json.dumps(res))
        return
    n = args.n
    zones = n ** 3
    U0 = torch.from_numpy(inputs.sod_planar(n)).to("cuda")

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    tol, guess, train_info = args.converged, None, None
    if args.learned_guess:
        from paper_1006_2146_gb300 import learned
        t0 = time.perf_counter()
        X, Y = learned.make_samples(learned.training_states(96), 96)
        guess, losses = learned.train(X, Y)
        torch.cuda.synchronize()
        train_info = {"samples": int(X.shape[0]), "train_s": time.perf_counter() - t0, "final_loss": losses[-1]}
        del X, Y
        if tol is None:
            tol = 1e-6 if args.fp32 else 1e-13

    # headline: timed region bracketed by barrier + synchronize
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    t0 = time.perf_counter()
    secs, prof, s, d, launches = run_config(ader, torch, n, args.order, args.form, args.solver, args.fp32,
                                            args.steps, args.warmup, stream, profile=True, state=U0, tol=tol,
                                            guess=guess)
    barrier()
    wall = time.perf_counter() - t0
    ck = clocks.stop()
    secs = max_over_ranks(secs, world, "cuda")
    value = job_throughput(zones, args.steps, world, secs)

    # dominant kernel roofline: FLOPs per zone x zones / mean launch time.  The plain kernels are bound by
    # the FP64 (or FP32) ALUs; the learned-guess kernel is a dense contraction on the tensor cores.
    fpz = flops_per_zone(args.order, args.form, args.solver, args.fp32)
    fpz["learned_guess"] = 2.0 * (52 * 128 + 128 * 128 + 128 * 25)       # the MLP's multiply-adds per zone
    kname, (kl, kms) = max(((k, v) for k, v in prof.items()), key=lambda kv: kv[1][1])
    k_avg = kms / kl / 1e3
    units = zones
    if kname == "learned_guess":      # the network runs only on the zones with slopes
        units = ader.ader_guess_count(s.h, stream)
    achieved = fpz[kname] * units / k_avg / 1e12 if kname in fpz else None
    sm_mhz = ck.get("sm_mhz") or 2070.0
    if kname == "learned_guess":
        bound, peak = "tensor", peaks().get("bf16_tflops", 1940.9)
        basis = "measured dense bf16 burst (MEASURED_PEAKS.json); FP16 operands run at the bf16 rate"
    else:
        bound, peak = "alu", alu_peak_tflops(args.fp32, 2070.0)
        basis = "derived: 152 SM x %s at 2070 MHz max clock" % (
            "128 FFMA/clk" if args.fp32 else "2 DFMA/clk (1.25 TFLOP/s nominal FP64)")
    total_ms = sum(v[1] for v in prof.values())
    roofline = {"bound": bound, "kernel": kname, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved else None,
                "traffic": traffic_per_launch(kname, args.order, args.form, args.fp32, zones),
                "peak_basis": basis,
                "flops_per_zone": fpz.get(kname), "zones_per_launch": units, "mean_launch_ms": k_avg * 1e3,
                "kernel_share": {k: round(v[1] / total_ms, 4) for k, v in prof.items()},
                "hbm": {"algorithmic_bytes_per_zone_update": 80,
                        "achieved_gbs": 80.0 * zones * args.steps / secs / 1e9,
                        "peak_gbs": peaks().get("hbm_gbs"), "frac": 80.0 * zones * args.steps / secs / 1e9 / peaks().get("hbm_gbs", 6658.3)}}
    guess_zones = ader.ader_guess_count(s.h, stream) if guess is not None else None
    s.close()
    del d

    # end-to-end through host memory: ader_step_host (H2D state, max_dt, step, D2H state) per step
    host = torch.from_numpy(inputs.sod_planar(n)).pin_memory().numpy()
    se = ader.Solver((n, n, n), order=args.order, form=args.form, solver=args.solver, fp32=args.fp32)
    for _ in range(2):
        ader.ader_step_host(se.h, host, None, 0.4)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ader.ader_step_host(se.h, host, None, 0.4)
    barrier()
    e2e_s = time.perf_counter() - t0
    se.close()
    e2e = {"value": zones * args.steps * world / e2e_s, "unit": "zone-updates/s",
           "h2d_bytes_per_step": 5 * 8 * zones, "d2h_bytes_per_step": 5 * 8 * zones + 8}

    variants = {}
    if not args.no_variants and rank == 0:
        vs = []
        for order in (2, 3, 4):
            vs.append(("fp64_modal_hll_o%d" % order, order, "modal", "hll", False))
            vs.append(("fp32_modal_hll_o%d" % order, order, "modal", "hll", True))
        vs += [("fp64_nodal_linearized_o3", 3, "nodal", "linearized", False),
               ("fp32_nodal_hll_o3", 3, "nodal", "hll", True)]
        vs = [v + (None, True) for v in vs]
        # the same step with a non-stiff source (uniform gravity): its cost in the predictor
        grav = ("gravity", (0.0, 0.0, -1.0))
        vs += [("fp64_nodal_hll_o3_gravity", 3, "nodal", "hll", False, grav, True),
               ("fp32_nodal_hll_o3_gravity", 3, "nodal", "hll", True, grav, True)]
        # the per-zone layout (face data of every zone through memory) beside the default tiles
        vs += [("fp32_nodal_hll_o3_per_zone_layout", 3, "nodal", "hll", True, None, False),
               ("fp32_modal_hll_o2_per_zone_layout", 2, "modal", "hll", True, None, False),
               ("fp64_nodal_hll_o3_per_zone_layout", 3, "nodal", "hll", False, None, False)]
        for name, order, form, solver, fp32, src, tiled in vs:
            try:
                vsecs, vprof, vs_, _, _ = run_config(ader, torch, n, order, form, solver, fp32, 3, 1, stream,
                                                     profile=True, state=U0, source=src, tiled=tiled)
                vs_.close()
                variants[name] = {"zone_updates_per_s": zones * 3 / vsecs, "ms_per_step": vsecs / 3 * 1e3,
                                  "kernel_ms": {k: round(v[1] / v[0], 3) for k, v in vprof.items()}}
            except Exception as exc:          # a variant that fails is reported, not hidden
                variants[name] = {"error": str(exc)[:200]}
        try:
            variants["dense_output_o3_nodal_fp64"] = dense_output_variant(ader, torch, stream, n, U0)
        except Exception as exc:
            variants["dense_output_o3_nodal_fp64"] = {"error": str(exc)[:200]}
        variants.update(learned_variants(ader, torch, n, U0, stream))
        variants.update(mhd_variants(ader, torch, stream))
        variants["learned_guess_mhd_ot_128"] = mhd_learned_evaluation(ader, torch, stream)
        try:
            variants["density_wave_convergence_fp64"] = convergence_variant(ader, torch)
        except Exception as exc:
            variants["density_wave_convergence_fp64"] = {"error": str(exc)[:200]}
        try:
            variants["vortex_tables_i_ii_fp64"] = vortex_tables(
                ader, torch, sizes=tuple(int(v) for v in args.vortex_sizes.split(",")))
        except Exception as exc:
            variants["vortex_tables_i_ii_fp64"] = {"error": str(exc)[:200]}
        if args.blast_symmetry:
            variants["blast_symmetry_fp64"] = blast_symmetry(ader, torch)
        variants["batched_64_problems_fp32"] = batched_variant(ader, torch, stream)
        variants["batched_512_small_problems_fp32"] = batched_variant(ader, torch, stream, count=512,
                                                                      sizes=(16, 24, 32))
        # SSP-RK of the same order and solver on the same GPU (Eq. 19), per step
        srk = ader.Solver((n, n, n), order=3, form="nodal", solver="hll")
        drk = U0.clone()
        dtv = 1e-4
        torch.cuda.synchronize()                        # the copy (current stream) before `stream` reads it
        with torch.cuda.stream(stream):
            srk.rk_step(drk, dtv, stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                srk.rk_step(drk, dtv, stream)
            e1.record(stream)
        torch.cuda.synchronize()
        rks = e0.elapsed_time(e1) / 1e3
        variants["fp64_ssprk3_hll_o3"] = {"zone_updates_per_s": zones * 3 / rks, "ms_per_step": rks / 3 * 1e3}
        srk.close()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, budget_s=15.0)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "zone-updates/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.fp32 else "f64",
                "data": "synthetic (seeded analytic Sod tube; no dataset)",
                "config": {"workload": "3D Euler Sod tube along (1,1,0), %d^3 periodic, order %d %s %s, CFL 0.4"
                                       % (n, args.order, args.form, args.solver.upper()),
                           "grid": n, "order": args.order, "form": args.form, "solver": args.solver,
                           "precision": "fp32 bulk + fp64 update" if args.fp32 else "fp64",
                           "predictor": ("converged, tol %g" % tol if tol else "fixed M-1 iterations") +
                                        (", learned initial guess" if guess is not None else ""),
                           "learned_guess_zones_per_step": guess_zones,
                           "l2": "state 671 MB > L2 129 MB (no flush needed)",
                           "parallelism": "independent problem per GPU" if world > 1 else "single GPU"},
                "roofline": roofline, "e2e": e2e, "gpu_launches": launches * args.steps,
                "launches_per_step": launches, "clocks": ck, "wall_s_timed": wall, "variants": variants}
        lg = variants.get("fp32_learned_guess_nodal_o3", {})
        if "zone_updates_per_s" in lg:
            line["fp32_learned_guess"] = {
                "zone_updates_per_s": lg["zone_updates_per_s"],
                "speedup_vs_fp64_plain": lg["zone_updates_per_s"] / value if not args.fp32 else None,
                "rel_l1_vs_fp64_converged_3steps": lg.get("rel_l1_vs_fp64_converged_3steps"),
                "mean_predictor_iterations": lg.get("mean_predictor_iterations")}
        rk = variants.get("fp64_ssprk3_hll_o3", {})
        if "zone_updates_per_s" in rk and not args.fp32 and args.order == 3 and args.solver == "hll":
            line["ader_vs_ssprk"] = {
                "ader_zone_updates_per_s": value, "ssprk3_zone_updates_per_s": rk["zone_updates_per_s"],
                "ader_over_ssprk_per_step": value / rk["zone_updates_per_s"],
                "paper_context": "Table V: ADER about 2x the SSP-RK speed at the same order (one CPU core)"}
        per_order = {}
        for o in (2, 3, 4):
            rec = {}
            for prec in ("fp64", "fp32"):
                vv = variants.get("%s_modal_hll_o%d" % (prec, o), {})
                if "zone_updates_per_s" in vv:
                    rec[prec + "_plain_modal"] = vv["zone_updates_per_s"]
            if rec:
                per_order["order%d" % o] = rec
        if "order3" in per_order and "zone_updates_per_s" in lg:
            per_order["order3"]["fp32_learned_guess_nodal"] = lg["zone_updates_per_s"]
        if per_order:
            line["per_order"] = per_order
        if train_info:
            line["learned_guess_training"] = train_info
        if cpu:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- oracle timings
def cpu_baseline(args, budget_s=15.0):
    """The FP64 oracle (numpy, as it stands) on a bounded sample of the same workload."""
    import numpy as np

    from oracle import scheme
    from paper_1006_2146_gb300 import inputs
    m = 32
    U = inputs.sod_planar(m)
    dx = (1.0 / m,) * 3
    t0, c0 = time.perf_counter(), time.process_time()
    steps = 0
    while time.perf_counter() - t0 < budget_s or steps == 0:
        dt = scheme.max_dt(U, dx, 0.4)
        U = scheme.ader_step(U, dx, dt, args.order, args.form, args.solver)
        steps += 1
    el = time.perf_counter() - t0
    threads = cores_used(time.process_time() - c0, el)
    return {"value": m ** 3 * steps / el, "unit": "zone-updates/s", "cores": threads, "host_cores": host_cores(),
            "kind": "oracle",
            "sample": "%d steps of the same scheme on a %d^3 Sod tube (numpy FP64 oracle, %.1f s)" % (steps, m, el)}


def reference_arm(args):
    """The oracle as it stands (numpy FP64) on the host cores: W untimed then K timed steps, each step one ADER
    step of the headline scheme on a bounded 32^3 sample of the same workload (rank 0 only)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import scheme
    from paper_1006_2146_gb300 import inputs
    m = 32
    U = inputs.sod_planar(m)
    dx = (1.0 / m,) * 3

    def step(U):
        dt = scheme.max_dt(U, dx, 0.4)
        return scheme.ader_step(U, dx, dt, args.order, args.form, args.solver)

    for _ in range(args.warmup):
        U = step(U)
    t0, c0 = time.perf_counter(), time.process_time()
    for _ in range(args.steps):
        U = step(U)
    el = time.perf_counter() - t0
    threads = cores_used(time.process_time() - c0, el)
    value = m ** 3 * args.steps / el
    cpu = {"value": value, "unit": "zone-updates/s", "cores": threads, "host_cores": host_cores(), "kind": "oracle",
           "sample": "%d timed steps (after %d untimed) of the same scheme on a %d^3 Sod tube (numpy FP64 "
                     "oracle, %.1f s)" % (args.steps, args.warmup, m, el)}
    line = {"metric": METRIC, "value": value, "unit": "zone-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "3D Euler Sod tube along (1,1,0), order %d %s %s (bounded %d^3 sample per "
                                   "step)" % (args.order, args.form, args.solver.upper(), m)},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "zone-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        reference_arm(a)
    else:
        gpu_arm(a)
