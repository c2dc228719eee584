"""Shared pieces of the GPU tests: building the library, comparing a context
against the FP64 oracle, and the tolerances.

Tolerances (written out here and used by every GPU force test):
The WCA force of one feature pair is steep: its logarithmic slope in r is
about 20-30 inside the cutoff.  A geometry error of delta (absolute, in the
nearest-point distance) changes a term's force by about |f'(r)| delta, which
relative to the term itself blows up near r_cut where f -> 0.  Each term k
therefore gets the scale s_k = |f_k| + sigma |f'(r_k)| (the force change
caused by a relative geometry perturbation of order one at the scale sigma),
and a particle's force error is measured against S_i = sum_k s_k (sums of
magnitudes, so cancellation between terms cannot hide an error):
    err_F(i) = |F_i - F_i^oracle| / S_i.
Torques use T_i = sum_k (|p_i - x_i| s_k + sigma |f_k|), energies
sigma * S_i.  The bars:
    FP64 mode:            err <= 1e-12
    FP32 and FP32 + two-sum:  err <= 1e-5   (relative 1e-5 on FP32 forces)
FP32 geometry with coordinates of order one carries errors of a few 1e-7,
i.e. a few 1e-7 / sigma relative to S_i; 1e-5 leaves a margin of ten or more.
Particles the oracle flags as having an edge pair within a decade of the
parallel-edge threshold are excluded (there the rule switches branch, and a
lower-precision evaluation may take the other one) and counted; every
parity test bounds their number to 1% of the particles.

A second, stricter measure relates each particle's error to its own net
force instead of its terms' scales:
    rel_F(i) = |F_i - F_i^oracle| / max(|F_i^oracle|, 1e-2 F_rms),
F_rms the root mean square net force over the particles with terms, and
the same for torques.  Where a particle's terms cancel this amplifies the
rounding of its terms: by the ratio of S_i to max(|F_i|, 1e-2 F_rms),
which reaches 1e3 or more for particles with many steep, nearly cancelling
terms.  FP64 rounds positions of size L (the box) and contact geometry of
order one to about 1e-16 of them; with that amplification the net-force
error of FP64 reaches a few 1e-12, so its bar is 1e-10 (measured worst:
2.2e-12 on the full-size batch).  It is reported for every case ("relF",
"relT") and bounded by RELTOL; it is skipped for states with overlapping
inner shapes (where a particle's terms are far above every net force and
no relative measure is meaningful).  Its denominators have a floor of
1e-12 of the particle's term scale, so that analytically zero quantities
(the torques of spheres) do not divide rounding by zero.
"""
from __future__ import annotations

import numpy as np

TOL = {0: 1e-12, 1: 1e-5, 2: 1e-5}
# bars of the net-force measure rel_F / rel_T (see above)
RELTOL = {0: 1e-10, 1: 1e-3, 2: 1e-5}
FLAGGED_MAX = 0.01        # largest fraction of particles excluded near the parallel band


def load_dem():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1607_02427_gb300 import dem
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return dem


def compare_forces(dem, system, precision, ref=None, **params):
    """Run one force evaluation; return (errors dict, ref, gpu outputs)."""
    import oracle
    if ref is None:
        ref = oracle.forces(system, par_eps=params.get("par_eps", oracle.DEFAULT_PAR_EPS))
    with dem.DEM(system, precision, **params) as d:
        f, t = d.forces()
        U, K, H = d.energy()
        W = d.virial()
        e = d.particle_energy()
        cnt = d.counters()
    out = dict(force=f, torque=t, U=U, W=W, energy=e, counts=cnt)
    return force_errors(system, ref, out), ref, out


def force_errors(system, ref, out):
    """Errors of GPU outputs (force, torque, energy per particle; U and W per
    replica; counts, or None) against the oracle's for the same system."""
    f, t, e, U, W = out["force"], out["torque"], out["energy"], out["U"], out["W"]
    ok = ref["flags"] == 0
    sig = system.sigma if system.sigma > 0 else 2 * max(sh["rounding"] for sh in system.shapes)
    S = np.maximum(ref["fscale"], 1e-300)
    T = np.maximum(ref["tscale"], 1e-300)
    errF = np.linalg.norm(f - ref["force"], axis=1) / S
    errT = np.linalg.norm(t - ref["torque"], axis=1) / T
    errU = np.abs(e - ref["energy"]) / np.maximum(sig * S, 1e-300)
    zero = ref["fscale"] == 0
    # particles without any term must get exactly zero
    zero_bad = (np.abs(f[zero]).max() if zero.any() else 0.0,
                np.abs(t[zero]).max() if zero.any() else 0.0)
    Rmax = max(float(np.max(np.linalg.norm(sh["verts"], axis=1))) for sh in system.shapes)
    sel = ok & ~zero
    Fn = np.linalg.norm(ref["force"], axis=1)
    Tn = np.linalg.norm(ref["torque"], axis=1)
    Frms = np.sqrt(np.mean(Fn[~zero] ** 2)) if (~zero).any() else 0.0
    Trms = np.sqrt(np.mean(Tn[~zero] ** 2)) if (~zero).any() else 0.0
    dF = np.maximum(np.maximum(Fn, 1e-2 * Frms), 1e-12 * S)
    dT = np.maximum(np.maximum(Tn, 1e-2 * Trms), 1e-12 * T)
    relF = np.linalg.norm(f - ref["force"], axis=1) / np.maximum(dF, 1e-300)
    relT = np.linalg.norm(t - ref["torque"], axis=1) / np.maximum(dT, 1e-300)
    errs = {
        "relF": float(relF[sel].max()) if sel.any() else 0.0,
        "relT": float(relT[sel].max()) if sel.any() else 0.0,
        "F": float(errF[ok & ~zero].max()) if (ok & ~zero).any() else 0.0,
        "T": float(errT[ok & ~zero].max()) if (ok & ~zero).any() else 0.0,
        "U": float(errU[ok & ~zero].max()) if (ok & ~zero).any() else 0.0,
        "zero": max(zero_bad),
        "flagged": int((~ok).sum()),
        "n": int(len(ok)),
        "normF": float(np.linalg.norm(f - ref["force"]) / max(np.linalg.norm(ref["force"]), 1e-300)),
    }
    # per-replica totals
    wscale = np.array([(2 * Rmax + 2 * sig) * ref["fscale"][sl].sum() + 1e-300
                       for sl in system.replica_slices()])
    Wref = np.stack([[v[0, 0], 0.5 * (v[0, 1] + v[1, 0]), 0.5 * (v[0, 2] + v[2, 0]), v[1, 1],
                      0.5 * (v[1, 2] + v[2, 1]), v[2, 2]] for v in ref["virial"]])
    errs["W"] = float((np.abs(W - Wref).max(1) / wscale).max())
    uscale = np.array([sig * ref["fscale"][sl].sum() + 1e-300 for sl in system.replica_slices()])
    errs["Utot"] = float((np.abs(U - ref["U"]) / uscale).max())
    cnt = out.get("counts")
    errs["counts"] = None if cnt is None else (cnt, ref["counts"].sum(0))
    return errs


def report(what, errs):
    """Append one line of measured errors to $DEM_PARITY_REPORT (if set)."""
    import json
    import os
    path = os.environ.get("DEM_PARITY_REPORT")
    if path:
        row = {k: v for k, v in errs.items() if k != "counts"}
        if errs["counts"] is not None:
            cnt, rc = errs["counts"]
            row["gpu_counts"] = [int(x) for x in cnt[:3]]
            row["oracle_counts"] = [int(x) for x in rc]
        with open(path, "a") as fh:
            fh.write(json.dumps({"case": what, **row}) + "\n")


def assert_parity(errs, precision, what="", flagged_max=FLAGGED_MAX, rel=True):
    report(what, errs)
    tol = TOL[precision]
    for k in ("F", "T", "U", "W", "Utot"):
        assert errs[k] <= tol, f"{what}: {k} error {errs[k]:.3e} > {tol:.0e} ({errs})"
    for k in (("relF", "relT") if rel else ()):
        assert errs[k] <= RELTOL[precision], \
            f"{what}: {k} error {errs[k]:.3e} > {RELTOL[precision]:.0e} ({errs})"
    assert errs["flagged"] <= flagged_max * errs["n"], \
        f"{what}: {errs['flagged']} of {errs['n']} particles flagged near the parallel band"
    assert errs["zero"] == 0.0, f"{what}: non-zero force on a particle without terms"
    if errs["counts"] is None:
        return
    cnt, rc = errs["counts"]
    # ordered pairs on the GPU, unordered in the oracle
    assert cnt[0] == 2 * rc[0], f"{what}: pairs in range {cnt[0]} vs 2 x {rc[0]}"
    assert cnt[1] == 2 * rc[1], f"{what}: feature pairs {cnt[1]} vs 2 x {rc[1]}"
    if precision == 0:
        assert cnt[2] == 2 * rc[2], f"{what}: contributing terms {cnt[2]} vs 2 x {rc[2]}"
    else:
        assert abs(cnt[2] - 2 * rc[2]) <= max(2, 1e-3 * rc[2]), f"{what}: terms {cnt[2]} vs {rc[2]}"
