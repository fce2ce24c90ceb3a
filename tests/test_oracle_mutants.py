"""Planted mistakes: every plausible slip in the oracle must trip a pin.

Each mutant is a copy of ``oracle/impact_oracle.c`` with one mistake planted
(a transposed operand, a flipped sign, a dropped factor, an off-by-one, a
wrong branch, ...), compiled with gcc on the CPU and run against the pins of
``oracle_pins.py`` in a child process. The test fails if any mutant passes
all pins, which would mean the pins cannot tell that mistake from the truth.
"""

import os
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

MUTANTS = {
    "A transposed": [("p->A[d * n + k] * xlo[k]", "p->A[k * n + d] * xlo[k]"),
                     ("p->A[d * n + k] * xhi[k]", "p->A[k * n + d] * xhi[k]")],
    "B transposed": [("p->B[d * p->m + k]", "p->B[k * p->n + d]")],
    "offset c dropped": [("double off = p->c ? p->c[d] : 0.0;", "double off = 0.0;")],
    "sign of (c - m)": [("double a = (c - m) / s;", "double a = (m - c) / s;")],
    "sigma read as variance": [("double a = (c - m) / s;", "double a = (c - m) / (s * s);"),
                               ("double b = (e - m) / s;", "double b = (e - m) / (s * s);")],
    "factor 1/2 dropped": [("return 0.5 * (erfc(a * M_SQRT1_2) - erfc(b * M_SQRT1_2));",
                            "return (erfc(a * M_SQRT1_2) - erfc(b * M_SQRT1_2));")],
    "straddle branch sign": [("- 0.5 * erfc(b * M_SQRT1_2);", "- 0.5 * erfc(-b * M_SQRT1_2);")],
    "no clamp for up": [("oracle_phi_diff(c, e, clamp(mid, m_lo[d], m_hi[d]), s)",
                         "oracle_phi_diff(c, e, mid, s)")],
    "no clamp for the sink": [("oracle_phi_diff(p->lo[d], p->hi[d], clamp(mid, m_lo[d], m_hi[d]), s)",
                               "oracle_phi_diff(p->lo[d], p->hi[d], mid, s)")],
    "mid of target wrong": [("double mid = 0.5 * (c + e);", "double mid = c;")],
    "lo takes max": [("l_t *= g_a < g_b ? g_a : g_b;", "l_t *= g_a < g_b ? g_b : g_a;")],
    "edge off by one": [("return p->lo[d] + (double)i * h;", "return p->lo[d] + (double)(i + 1) * h;")],
    "Fortran cell order": [("for (int k = d + 1; k < p->n; ++k) stride *= p->cells[k];",
                            "for (int k = 0; k < d; ++k) stride *= p->cells[k];")],
    "wrong input for row": [("int j = (int)(row % p->n_inputs);",
                             "int j = (int)((row + 1) % p->n_inputs);")],
    "cos range misses extremum": [("(long)ceil(a / M_PI)", "(long)ceil(a / M_PI) + 1")],
    "cos and sin swapped": [("cos_range(xlo[2], xhi[2], &cl, &ch);",
                             "sin_range(xlo[2], xhi[2], &cl, &ch);")],
    "theta input sign": [("m_hi[2] = xhi[2] + om;", "m_hi[2] = xhi[2] - om;")],
    "sink_lo from the min": [("in_max *= G_max;", "in_max *= G_a < G_b ? G_a : G_b;")],
    "sink bounds swapped": [("*sink_lo = 1.0 - in_max;", "*sink_lo = 1.0 - in_min;"),
                            ("*sink_up = 1.0 - in_min;", "*sink_up = 1.0 - in_max;")],
    "trunc sums lo": [("else neumaier_add(&s, &comp, up[t]);",
                       "else neumaier_add(&s, &comp, lo[t]);")],
    "region lo takes max": [("b_lo *= r_a < r_b ? r_a : r_b;", "b_lo *= r_a < r_b ? r_b : r_a;")],
    "region box one cell short": [("double right = oracle_edge(p, d, last[d] + 1);",
                                   "double right = oracle_edge(p, d, last[d]);")],
    "region centre not clamped": [("clamp(centre, m_lo[d], m_hi[d])", "centre")],
    "sink left out of A": [("out[2] = sl + x_lo;", "out[2] = x_lo;"),
                           ("out[3] = su + x_up;", "out[3] = x_up;")],
    "region sums take up for lo": [("{ r_lo += lo[t]; r_up += up[t]; }",
                                    "{ r_lo += up[t]; r_up += up[t]; }")],
    "labels: target wins": [("if (in && avoid) lab = ORACLE_AVOID;\n            else if (in && lab == ORACLE_FREE) lab = ORACLE_TARGET;",
                             "if (in && !avoid) lab = ORACLE_TARGET;\n            else if (in && lab == ORACLE_FREE) lab = ORACLE_AVOID;")],
    "cell centre off by half": [("return 0.5 * (oracle_edge(p, d, i) + oracle_edge(p, d, i + 1));",
                                 "return oracle_edge(p, d, i);")],
    "cell_of closes the cell": [("if (y < oracle_edge(p, d, i + 1)) return i;",
                                 "if (y <= oracle_edge(p, d, i + 1)) return i;")],
    "mc box ends swapped": [("b[d] = oracle_cell_of(p, d, w + m_hi[d]);",
                             "b[d] = oracle_cell_of(p, d, w - m_hi[d]);")],
    "mc lo without the single test": [("if (single) ++lo[t];", "++lo[t];")],
    "mc sink_up counts leaving whole": [("if (!inside) ++*sink_up;", "if (outside) ++*sink_up;")],
    "mc dropped mass from lo": [("else dropped += up[t];", "else dropped += lo[t];")],
    "ties dropped": [("if (up[t] >= p->cutoff) ++cnt;", "if (up[t] > p->cutoff) ++cnt;"),
                     ("if (up[t] >= p->cutoff) {", "if (up[t] > p->cutoff) {")],
}

RUNNER = r"""
import sys
sys.path[:0] = [{root!r}, {tests!r}]
import numpy as np
import oracle, oracle_pins as P
orc = oracle.Oracle({lib!r})
try:
    P.pin_phi_library(orc, trials=60)
    P.pin_edges_telescoping(orc)
    P.pin_closed_form_1d(orc)
    P.pin_bruteforce_2d(orc, cells_per_dim=5, rows=[0, 31, 112, 200])
    P.pin_unicycle_image(orc)
    P.pin_degenerate(orc)
    P.pin_tie_kept(orc)
    for prob, rows in P.coupled_cases():
        P.pin_mc_containment(orc, prob, rows[:2], samples=12)
        P.pin_invariants(orc, prob, rows[:2])
    for k in (0, 2):
        prob, rows = P.coupled_cases()[k]
        P.pin_separable_sum(orc, prob, rows[:2])
    from paper_2401_03555_gb300 import workloads as W
    for prob in (W.bas_4d(eta_scale=2.0), W.unicycle_3d(nx=8, ny=8, nth=6)):
        P.pin_noise_sampling(orc, prob, W.sample_rows(prob, 1, seed=9, include_boundary=False)[0],
                             draws=60000)
    P.pin_region_labels(orc)
    P.pin_region_containment(orc, samples=6)
    P.pin_region_box_exact_separable(orc)
    P.pin_region_reductions(orc)
    P.pin_mc_cell_of(orc)
    P.pin_mc_point_images(orc, S=6000)
    P.pin_mc_box_images(orc, S=6000)
    P.pin_mc_counting(orc, S=600)
except AssertionError as e:
    print("CAUGHT", repr(e)[:200])
    sys.exit(3)
sys.exit(0)
"""


def _mutate(src, subs):
    for old, new in subs:
        assert src.count(old) == 1, f"mutation anchor not unique/present: {old!r}"
        src = src.replace(old, new)
    return src


def _run(name, subs, tmp):
    src = _mutate(oracle.source_text(), subs)
    lib = oracle.compile_variant(src, os.path.join(tmp, name.replace(" ", "_")))
    code = RUNNER.format(root=ROOT, tests=HERE, lib=lib)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    return name, r.returncode, (r.stdout + r.stderr)[-300:]


def test_unmutated_source_passes_runner():
    with tempfile.TemporaryDirectory() as tmp:
        name, rc, out = _run("identity", [], tmp)
    assert rc == 0, out


def test_every_planted_mistake_is_caught():
    with tempfile.TemporaryDirectory() as tmp:
        with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
            results = list(ex.map(lambda kv: _run(kv[0], kv[1], tmp), MUTANTS.items()))
    survivors = [(n, out) for n, rc, out in results if rc == 0]
    assert not survivors, f"mutants not caught by any pin: {survivors}"
