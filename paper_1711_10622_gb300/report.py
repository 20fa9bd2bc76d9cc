"""The paper's performance model evaluated on measured GSpMV timings (Section 2.3).

The paper predicts the gain of solving m right-hand sides together from the memory traffic of CRS
GSpMV and turns it into a time-step and an overall simulation speedup. Given measured GSpMV times
t(m) on one GPU, this module puts the measured gain m t(1) / t(m) beside the model's
5m / (2m + 3) (Eq. mem_GSpMV_compact) and the full form with the operator's C = nnz / n
(Eq. mem_GSpMV_full), and evaluates the step gain (Eq. est2_1) and the overall speedup P_m
(Eq. est2) from the measured gain at the paper's theta and beta values.
"""

from __future__ import annotations

# Context quoted with the hardware the paper names (not a target for this GPU).
PAPER_HEADLINE = {
    "claim": "speedup of DNS/LES by simultaneous modelling of several flow states: about 1.5-2x",
    "hardware": "Lomonosov (2x Intel Xeon X5570 per node, QDR InfiniBand) and Lomonosov-2 "
    "(1x Intel Xeon E5-2697v3 per node, FDR InfiniBand)",
    "where": "Abstract, Sections 4.2-4.3 and Conclusions",
}


def compact_gain(m: int) -> float:
    """Traffic gain of GSpMV with m vectors for C >> 1: 5m / (2m + 3)."""
    return 5.0 * m / (2.0 * m + 3.0)


def full_gain(m: int, C: float) -> float:
    """Traffic gain with C nonzeros per row: m(5C + 3) / (2m(C + 1) + 3C + 1)."""
    return m * (5.0 * C + 3.0) / (2.0 * m * (C + 1.0) + 3.0 * C + 1.0)


def step_gain(theta: float, solver_gain: float) -> float:
    """m t_1 / t_m for a step whose solver share is theta (the rest scales with m)."""
    return 1.0 / (theta / solver_gain + 1.0 - theta)


def overall_speedup(m: int, beta: float, step: float) -> float:
    """P_m = (1 + beta) / (m + beta) * m t_1 / t_m."""
    return (1.0 + beta) / (m + beta) * step


def estimate_table(times_us: dict, n: int, nnz: int, thetas=(0.80, 0.85), betas=(5.0, 20.0)) -> dict:
    """Table of the paper's estimate on measured GSpMV times {m: microseconds} (m = 1 required)."""
    if 1 not in times_us:
        raise ValueError("the m = 1 time is needed for the measured gain")
    C = nnz / n
    t1 = times_us[1]
    rows = []
    for m in sorted(times_us):
        g = m * t1 / times_us[m]
        row = {
            "m": m,
            "t_us": times_us[m],
            "measured_gain": g,
            "model_compact": compact_gain(m),
            "model_full": full_gain(m, C),
        }
        for th in thetas:
            sg = step_gain(th, g)
            row[f"step_gain_theta{th:.2f}"] = sg
            for be in betas:
                row[f"P_theta{th:.2f}_beta{be:g}"] = overall_speedup(m, be, sg)
        rows.append(row)
    best = {}
    for th in thetas:
        for be in betas:
            key = f"P_theta{th:.2f}_beta{be:g}"
            r = max(rows, key=lambda r: r[key])
            best[key] = {"m": r["m"], "P": r[key]}
    return {"C": C, "rows": rows, "best_m": best, "paper_headline": PAPER_HEADLINE}
