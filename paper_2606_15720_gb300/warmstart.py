"""Learned warm start of steady solves.

Training data are the converged fields of cases the solver itself ran:
for every cell, the feature vector of ``ugks_mlp_features`` (Mach, log10 Kn,
centroid, wall distance) and the thirteen-moment fields of
``ugks_moments13`` (rho, U, T, deviatoric stress, heat flux).  The network is
trained and evaluated by the library's kernels (``WarmStartNet``); this
module only gathers arrays and drives the calls.
"""
from __future__ import annotations

import time
from typing import Optional, Sequence

import numpy as np

from . import ugks as U
from .inputs import BC_FARFIELD


def converge(solvers: Sequence["U.Solver"], tol: float = 1e-6, max_steps: int = 200_000, check_every: int = 200,
             batch: Optional["U.Batch"] = None):
    """Steps until the density residual R_rho of every case is below tol
    (checked every ``check_every`` steps).  Returns the steps each case took
    (None where max_steps was reached first or the case became non-physical,
    which ends its stepping).  With ``batch`` the cases are stepped together
    by its graph launches; converged cases keep stepping until all are done
    (their fields no longer change at that tolerance)."""
    steps = [None] * len(solvers)
    failed = [False] * len(solvers)
    done = 0
    while done < max_steps and any(s is None and not f for s, f in zip(steps, failed)):
        if batch is not None:
            batch.step(check_every)
        else:
            for i, s in enumerate(solvers):
                if steps[i] is None and not failed[i]:
                    s.step(check_every)
        done += check_every
        for i, s in enumerate(solvers):
            if steps[i] is not None or failed[i]:
                continue
            try:
                if s.residual()[0] < tol:
                    steps[i] = done
            except U.UGKSError:
                failed[i] = True
    return steps


def time_to_steady(solver: "U.Solver", tol: float = 1e-6, max_steps: int = 200_000, check_every: int = 200):
    """(steps, seconds) until R_rho < tol, the seconds on the host clock
    around the stepping (each check synchronises)."""
    t0 = time.perf_counter()
    steps = converge([solver], tol, max_steps, check_every)[0]
    return steps, time.perf_counter() - t0


def training_set(net: "U.WarmStartNet", solvers, meshes, machs, kns):
    """Stacks (features, fields) of every cell of every converged case."""
    X, Y = [], []
    for s, m, ma, kn in zip(solvers, meshes, machs, kns):
        X.append(net.features(m, ma, kn))
        Y.append(s.moments13().astype(np.float32))
    return np.concatenate(X), np.concatenate(Y)


def freestream_fields(mesh) -> np.ndarray:
    """(rho, U[dim], T) of the mesh's first far-field condition."""
    bcs = [b for b in mesh.bc if b.type == BC_FARFIELD]
    b = bcs[0] if bcs else mesh.bc[1]
    return np.array([b.rho, *b.u[:mesh.dim], b.T], dtype=np.float64)


def cylinder_case(mach: float, kn: float, cells: int, nvx: Optional[int], seed: int, family: str = "shakhov"):
    """One cylinder case of a warm-start family.

    family "shakhov": a Shakhov gas (Pr 2/3, omega 0.81) started from the
    freestream, far-field lateral edges (this family's flows, Ma <= 3, keep
    the bow shock clear of them) and an nvx^2 midpoint velocity grid on
    [-v, v]^2, v = max(U_inf + 4, 3.5 sqrt(T_stag)).

    family "batch": a case of the cylinder batch workload's kind (Ma 2-8):
    BGK (omega 0.81) with Venkatakrishnan's K_v = 1, outflow lateral edges,
    the potential-flow start, and (nvx None) the batch's grid rule, nvx =
    clip(ceil(2 v / 0.7), 20, 48)."""
    import math
    from . import inputs as I
    u_inf = mach * math.sqrt(5.0 / 6.0)
    vmax = max(u_inf + 4.0, 3.5 * math.sqrt(1.0 + mach * mach / 3.0))
    if family == "shakhov":
        mesh = I.cylinder_tri_mesh(cells, seed=seed, mach=mach, lateral="farfield")
        grid = I.midpoint_grid(nvx, -vmax, vmax, 2)
        gas = I.Gas(model="shakhov", K=0, Pr=2.0 / 3.0, omega=0.81, mu_ref=I.mu_ref_from_kn(kn, 0.81), cfl=0.8)
        W0 = I.prim_to_conservative(I.uniform_primitives(mesh, 1.0, mesh.bc[1].u, 1.0), 2, 0)
    elif family == "batch":
        mesh = I.cylinder_tri_mesh(cells, seed=seed, mach=mach)
        n = nvx if nvx else int(min(48, max(20, math.ceil(2.0 * vmax / 0.7))))
        grid = I.midpoint_grid(n, -vmax, vmax, 2)
        gas = I.Gas(model="bgk", K=0, Pr=1.0, omega=0.81, mu_ref=I.mu_ref_from_kn(kn, 0.81), cfl=0.8, venkat_K=1.0)
        W0 = I.prim_to_conservative(I.cylinder_potential_primitives(mesh, mesh.bc[1].u[0]), 2, 0)
    else:
        raise ValueError("family must be 'shakhov' or 'batch'")
    return mesh, grid, gas, W0


def rel_linf(W, W_ref):
    """Per-field relative L-infinity difference max_i |W - W_ref| / max_i |W_ref|."""
    return (np.abs(W - W_ref).max(0) / np.maximum(np.abs(W_ref).max(0), 1e-300)).tolist()


def experiment(train, held_out, cells: int, nvx: Optional[int], width: int = 256, hidden_layers: int = 6,
               schedule=((200, 1e-3), (200, 3e-4), (100, 1e-4)), batch: int = 512, tol: float = 1e-6,
               ref_tol: Optional[float] = None, check_every: int = 200, max_steps: int = 200_000, seed: int = 0,
               log=None, family: str = "shakhov") -> dict:
    """Trains the warm start on converged cases and measures what it gains.

    train, held_out: sequences of (Mach, Kn).  The training cases run together
    in one batch (CUDA graph) to R_rho < tol; the network is trained on their
    per-cell features and thirteen-moment fields.  Every held-out case (a new
    mesh) is then solved twice to R_rho < tol, from the freestream and from
    the warm start, and the steps and host seconds of both (the warm start's
    own set-up included) are returned.  With ref_tol the freestream solve
    continues to R_rho < ref_tol as the reference; both converged fields and
    both starting states are compared with it (per-field relative L-inf), and
    the warm solve also records when every field is at least as close to the
    reference as the freestream solve was at R_rho < tol (equal accuracy).
    The warm solve's checks then also read W every check_every steps.
    family selects the kind of case (cylinder_case); training cases that do
    not reach tol within max_steps are left out of the training set."""
    def say(*a):
        if log:
            log(" ".join(str(x) for x in a))

    out = {"train": [list(t) for t in train], "held_out": [list(t) for t in held_out], "cells": cells,
           "nvx": nvx, "family": family, "tol": tol, "ref_tol": ref_tol,
           "network": f"{hidden_layers}x{width} tanh, BF16/FP32-acc"}
    cases = [cylinder_case(ma, kn, cells, nvx, seed=1000 + i, family=family) for i, (ma, kn) in enumerate(train)]
    t0 = time.perf_counter()
    with U.Batch([c[0] for c in cases], [c[1] for c in cases], [c[2] for c in cases], [c[3] for c in cases],
                 storage="f32") as b:
        steps = converge(b.cases, tol, max_steps, check_every, batch=b)
        out["train_converge"] = {"steps": steps, "seconds": time.perf_counter() - t0}
        say("training cases converged", steps, round(time.perf_counter() - t0, 1), "s")
        D = cases[0][0].dim
        net = U.WarmStartNet(6, 2 * D + 2 + D * (D + 1) // 2, width=width, hidden_layers=hidden_layers, seed=seed)
        keep = [i for i, n in enumerate(steps) if n is not None]
        X, Y = training_set(net, [b.cases[i] for i in keep], [cases[i][0] for i in keep],
                            [train[i][0] for i in keep], [train[i][1] for i in keep])
    net.fit_scaling(X, Y)
    t0 = time.perf_counter()
    losses = []
    for i, (epochs, lr) in enumerate(schedule):
        losses.append(net.train(X, Y, epochs=epochs, batch=batch, lr=lr, seed=seed + i))
        say("epochs", epochs, "lr", lr, "loss", losses[-1])
    secs = time.perf_counter() - t0
    epochs = sum(e for e, _ in schedule)
    # tensor-core work: forward, data gradient and weight gradient GEMMs of
    # every layer (padded widths, the first layer has no data gradient)
    pad = lambda n: (n + 15) // 16 * 16  # noqa: E731
    sizes = [pad(n) for n in net.sizes]
    macs = sum(a * b for a, b in zip(sizes[:-1], sizes[1:]))
    flops = 2.0 * (3 * macs - sizes[0] * sizes[1]) * X.shape[0] * epochs
    out["training"] = {"samples": int(X.shape[0]), "epochs": epochs, "batch": batch,
                       "schedule": [list(s) for s in schedule], "loss": losses, "seconds": secs,
                       "gemm_tflops": flops / secs / 1e12}
    out["cases"] = []
    for j, (ma, kn) in enumerate(held_out):
        mesh, grid, gas, W0 = cylinder_case(ma, kn, cells, nvx, seed=5000 + j, family=family)
        rec = {"mach": ma, "kn": kn, "n_cells": int(mesh.n_cells)}
        W_ref = None
        with U.Solver(mesh, grid, gas, W0, storage="f32") as s:
            W_free = s.moments()
            n, sec = time_to_steady(s, tol, max_steps, check_every)
            rec["freestream"] = {"steps": n, "seconds": sec}
            if n is None:
                # non-physical or not converged within max_steps: no reference to compare with
                say("held-out", ma, kn, "plain start did not reach tol")
                out["cases"].append(rec)
                continue
            W_plain = s.moments()
            if ref_tol:
                if converge([s], ref_tol, max_steps, check_every)[0] is None:
                    rec["reference_not_reached"] = True
                try:
                    W_ref = s.moments()
                    e_plain = rel_linf(W_plain, W_ref)
                except U.UGKSError:
                    W_ref = None
        with U.Solver(mesh, grid, gas, W0, storage="f32") as s:
            t0 = time.perf_counter()
            nf = net.warm_start(s, mesh, ma, kn, freestream_fields(mesh))
            setup = time.perf_counter() - t0
            W_warm0 = s.moments()
            t0 = time.perf_counter()
            done, n_res, sec_res, n_acc, sec_acc, W_warm = 0, None, None, None, None, None
            while done < max_steps and (n_res is None or (W_ref is not None and n_acc is None)):
                s.step(check_every)
                done += check_every
                try:
                    r = s.residual()[0]
                except U.UGKSError:
                    rec["warm_non_physical_by_step"] = done
                    break

                if n_res is None and r < tol:
                    n_res, sec_res, W_warm = done, time.perf_counter() - t0 + setup, s.moments()
                if W_ref is not None and n_acc is None:
                    e = rel_linf(s.moments(), W_ref)
                    if all(a <= b for a, b in zip(e, e_plain)):
                        n_acc, sec_acc = done, time.perf_counter() - t0 + setup
            rec["warm"] = {"steps": n_res, "seconds": sec_res, "setup_seconds": setup, "fallback_cells": nf}
        if "warm_non_physical_by_step" in rec:
            # fallback: the plain start, after the steps and seconds lost on the warm one
            lost_steps, lost_sec = rec["warm_non_physical_by_step"], time.perf_counter() - t0 + setup
            with U.Solver(mesh, grid, gas, W0, storage="f32") as s:
                n, sec = time_to_steady(s, tol, max_steps, check_every)
                W_warm = s.moments() if n is not None else None
            n_res = lost_steps + n if n is not None else None
            sec_res = lost_sec + sec if n is not None else None
            rec["warm"] = {"steps": n_res, "seconds": sec_res, "setup_seconds": setup, "fallback_cells": nf,
                           "restarted_from_plain_start": True}
            n_acc, sec_acc = n_res, sec_res     # the plain solve's own accuracy
        if rec["freestream"]["steps"] and n_res:
            rec["step_ratio"] = rec["freestream"]["steps"] / n_res
            rec["time_ratio"] = rec["freestream"]["seconds"] / sec_res
            rec["converged_difference"] = rel_linf(W_warm, W_plain)
        if W_ref is not None:
            rec["error_vs_reference"] = {"freestream_start": e_plain,
                                         "warm_start": rel_linf(W_warm, W_ref) if W_warm is not None else None}
            rec["initial_error_vs_reference"] = {"freestream": rel_linf(W_free, W_ref),
                                                 "warm": rel_linf(W_warm0, W_ref)}
            rec["warm_equal_accuracy"] = {"steps": n_acc, "seconds": sec_acc}
            if n_acc and rec["freestream"]["steps"]:
                rec["equal_accuracy_step_ratio"] = rec["freestream"]["steps"] / n_acc
                rec["equal_accuracy_time_ratio"] = rec["freestream"]["seconds"] / sec_acc
        say("held-out", ma, kn, rec)
        out["cases"].append(rec)
    net.close()
    return out
