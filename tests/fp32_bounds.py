"""Bounds of the FP32-compensated outputs against the binary64 oracle, shared
by the GPU parity tests (the bounds are stated in test_parity_gpu.py's module
doc), and the per-sample proof that a brake-onset disagreement under the TTC
trigger is a rounding tie."""
import numpy as np

import aeb_inputs as ai

U32 = 2.0 ** -24
R_MAX = 10.0  # bound on |dv/dt| [m/s^2]


def lead_speed(m, t):
    if m.lead_decel > 0.0:
        return np.where(t >= m.lead_v0 / m.lead_decel, 0.0, m.lead_v0 - m.lead_decel * t)
    return np.full_like(np.asarray(t, dtype=np.float64), m.lead_v0)


def trigger_eps(m, rec, j, d0, k):
    t = k * m.dt
    xl = float(lead_pos(m, np.float64(t))) if m.lead else 0.0
    vl = float(lead_speed(m, np.float64(t))) if m.lead else 0.0
    return 2.0 ** -21 * (abs(rec["gap_meas"][j]) + abs(rec["thr_closing"][j]) + abs(rec["x"][j]) +
                         abs(d0) + abs(xl) + abs(m.ttc_thr) * abs(vl)) + 18 * U32 * m.perc_sigma


def resolve_onset_ties(oracle_mod, m, p, rows, got, exp):
    """Samples whose brake onset differs between the kernel and the oracle:
    prove each one a trigger tie (see the module doc) and replace its oracle
    outputs by those of the oracle run with the trigger forced to the kernel's
    step.  Returns the new oracle outputs and (tie count, worst |margin|/eps)."""
    on32, on64 = got["n_onset"], exp["n_onset"]
    idx = np.nonzero(on32 != on64)[0]
    if len(idx) == 0:
        return exp, (0, 0.0)
    assert m.trigger == ai.TRIGGER_TTC, "onset step must match in immediate mode"
    exp = {k: v.copy() for k, v in exp.items()}
    perc = m.perc_sigma > 0 or m.perc_drop > 0 or m.perc_latency > 0
    lat = oracle_mod.steps_to_reach(m.perc_latency, m.dt) if perc else 0
    n_max = oracle_mod.steps_to_reach(m.t_max, m.dt)
    worst = 0.0
    for i in idx:
        i = int(i)
        row = int(rows[i])
        nd = oracle_mod.steps_to_reach(float(p["t_delay"][i]), m.dt)
        t32 = int(on32[i]) - lat - nd if on32[i] >= 0 else None
        t64 = int(on64[i]) - lat - nd if on64[i] >= 0 else None
        d0 = float(p["d0"][i])
        if t64 is None or (t32 is not None and t32 < t64):
            # the kernel fired at t32 where the oracle did not: a tie at t32
            _, rec = oracle_mod.rollout_probe(m, p, i, row=row, force=-2, lo=t32, hi=t32 + 1)
            assert rec["reading"][0] >= 0, (i, "trigger not tested at the kernel's step")
            # (the kernel's dropout decision is the oracle's, exactly)
            assert rec["reading"][0] == 1, (i, "kernel fired without a reading")
            margin = rec["gap_meas"][0] - rec["thr_closing"][0]
            eps = trigger_eps(m, rec, 0, d0, t32)
            assert margin <= eps, (i, "not a tie: kernel fired early", margin, eps)
            worst = max(worst, abs(margin) / eps)
        else:
            # the oracle fired at t64; the kernel did not at t64 .. t32 - 1
            force = t32 if t32 is not None else -1
            hi = t32 if t32 is not None else n_max + 1
            _, rec = oracle_mod.rollout_probe(m, p, i, row=row, force=force, lo=t64, hi=hi)
            for j in range(hi - t64):
                if rec["reading"][j] != 1:
                    continue
                margin = rec["gap_meas"][j] - rec["thr_closing"][j]
                eps = trigger_eps(m, rec, j, d0, t64 + j)
                assert margin >= -eps, (i, "not a tie: kernel missed a clear trigger", t64 + j,
                                        margin, eps)
                if margin < 0:
                    worst = max(worst, -margin / eps)
        forced, _ = oracle_mod.rollout_probe(m, p, i, row=row,
                                             force=t32 if t32 is not None else -1)
        for k in exp:
            if k in forced:
                exp[k][i] = forced[k]
    return exp, (len(idx), worst)


def fp32_report(m, got, exp, ties=(0, 0.0)):
    """Compare FP32-compensated outputs with the binary64 ones (after
    resolve_onset_ties); return counts of tolerated disagreements and the worst
    errors, asserting the bounds of the module doc for every sample."""
    s32, s64 = got["status"], exp["status"]
    assert np.array_equal(got["n_onset"], exp["n_onset"]), "onset differs beyond the proven ties"
    flag_diff = s32 != s64
    rep = {"n": len(s32), "onset_ties": ties[0], "tie_margin_over_eps_max": ties[1],
           "flag_disagree": int(flag_diff.sum())}
    if flag_diff.any():
        # whichever path stopped must have stopped within 1e-3 m of the lead
        idx = np.nonzero(flag_diff)[0]
        stopped_gap = np.where(s64[idx] == 0, exp["gap"][idx], got["gap"][idx])
        assert np.all(np.abs(stopped_gap) < 1e-3), stopped_gap
    same = ~flag_diff
    st = same & (s64 == 0)
    rel = np.abs(got["x_ref"][st] - exp["x_ref"][st]) / np.maximum(np.abs(exp["x_ref"][st]), 1e-3)
    rep["x_ref_rel_max"] = float(rel.max()) if rel.size else 0.0
    rep["x_ref_rel_mean"] = float(rel.mean()) if rel.size else 0.0
    assert rep["x_ref_rel_max"] <= 1e-5, rep
    ct = same & (s64 == 1)
    if ct.any():
        vi = exp["v_imp"][ct]
        d0 = exp["x_ref"][ct]
        dv = np.abs(got["v_imp"][ct] - vi)
        dtc = np.abs(got["t_end"][ct] - exp["t_end"][ct])
        rep["v_imp_abs_max"] = float(dv.max())
        d0r = np.maximum(d0, 1e-3)  # (report only: a contact at x = 0 has no ratio)
        rep["contact_dt_x_v_over_d0_max"] = float((dtc * vi / d0r).max())
        rep["contact_dv_x_v_over_d0_max"] = float((dv * vi / d0r).max())
        assert np.all(dtc * vi <= 1e-5 * d0), rep
        assert np.all(dv * vi <= R_MAX * 1e-5 * d0), rep
    sp = same & (s64 == 0)
    dts = np.abs(got["t_end"][sp] - exp["t_end"][sp])
    rep["stop_t_end_abs_max"] = float(dts.max()) if dts.size else 0.0
    assert np.all(dts <= 1e-6 + 1e-6 * exp["t_end"][sp]), rep
    hz = same & (s64 == 2)
    assert np.array_equal(got["t_end"][hz], exp["t_end"][hz])
    # steps: equal, or one apart where the end falls on a step boundary
    dn = got["n_steps"].astype(np.int64) - exp["n_steps"].astype(np.int64)
    tie = same & (dn != 0)
    rep["n_steps_ties"] = int(tie.sum())
    assert np.all(np.abs(dn[tie]) == 1), "n_steps differ by more than one step"
    assert not np.any(tie & (s64 == 2)), "horizon step count differs"
    edge = np.minimum(got["n_steps"], exp["n_steps"]).astype(np.float64) * m.dt
    ts = tie & (s64 == 0)
    assert np.all(np.abs(exp["t_end"][ts] - edge[ts]) <= 1e-6 + 1e-6 * exp["t_end"][ts]), rep
    tc = tie & (s64 == 1)
    assert np.all(np.abs(exp["t_end"][tc] - edge[tc]) * exp["v_imp"][tc]
                  <= 1e-5 * exp["x_ref"][tc]), rep
    # x_raw, the paper's D_stop = x(t_stop)
    xr = np.abs(got["x_raw"] - exp["x_raw"])
    scale = np.maximum(np.abs(exp["x_raw"]), 1e-3)
    eq = same & (dn == 0)
    rep["x_raw_rel_max"] = float((xr[eq] / scale[eq]).max()) if eq.any() else 0.0
    assert rep["x_raw_rel_max"] <= 1e-5, rep
    v_lead = m.lead_v0 if m.lead else 0.0
    step_travel = np.where(s64 == 0, R_MAX * m.dt * m.dt,
                           m.dt * (np.abs(exp["v_imp"]) + v_lead + R_MAX * m.dt))
    assert np.all(xr[tie] <= 1e-5 * scale[tie] + step_travel[tie]), rep
    return rep


def lead_pos(m, t):
    """Closed-form position of the braking lead at times t (numpy)."""
    if m.lead_decel > 0.0:
        ts = m.lead_v0 / m.lead_decel
        return np.where(t >= ts, 0.5 * m.lead_v0 * ts, t * (m.lead_v0 - 0.5 * m.lead_decel * t))
    return t * m.lead_v0


def with_gap(out, p, m):
    """The gap to the lead where each rollout ended (inf without a lead)."""
    out = dict(out)
    if not m.lead:
        out["gap"] = np.full(len(out["x_ref"]), np.inf)
    else:
        out["gap"] = (p["d0"] + lead_pos(m, out["t_end"])) - out["x_ref"]
    return out
