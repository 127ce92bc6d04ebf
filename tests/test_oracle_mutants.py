"""The pins in test_oracle_pins.py are chosen so that a plausible mistake in
the oracle fails at least one of them.  This test plants such mistakes, one
at a time, in a copy of oracle/dwt_oracle.c (a flipped sign, a dropped factor,
a wrong or transposed index, another rounding rule, a wrong normalisation),
builds each copy with gcc, runs the pin suite against it in a subprocess
(DWTFUSE_ORACLE_LIB points the oracle at the copy), and requires the suite to
fail.  CPU only."""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "dwt_oracle.c")

# (name, text in dwt_oracle.c, replacement); each text occurs exactly once.
MUTANTS = [
    ("d4 g sign", "g[1] = -h[2];", "g[1] = h[2];"),
    ("d4 h index", "h[i + 2] = (3.0 - 2.0 * i - r3) / den;", "h[i + 2] = (3.0 - 2.0 * i + r3) / den;"),
    ("haar forward detail sign", "wt[1] = detail ? -0.5 : 0.5;", "wt[1] = detail ? 0.5 : -0.5;"),
    ("haar forward scale", "wt[0] = 0.5;", "wt[0] = 1.0;"),
    ("haar inverse sign", "wt[1] = (n % 2 == 0) ? 1.0 : -1.0;", "wt[1] = (n % 2 == 0) ? -1.0 : 1.0;"),
    ("d4 forward wrap index (Eq. 5-6)", "idx[2 + m] = m;", "idx[2 + m] = m + 1;"),
    ("d4 inverse table t", "const double t[4] = {w->h[2], w->g[2], w->h[0], w->g[0]};",
     "const double t[4] = {w->h[0], w->g[2], w->h[2], w->g[0]};"),
    ("d4 inverse wrap index (Eq. 13)", "idx[2 + k] = (N - 1) * k;", "idx[2 + k] = (N - 2) * k;"),
    ("d4 inverse interior index (Eq. 15)", "idx[2 + k] = i + half + k;", "idx[2 + k] = i + half - k;"),
    ("LL gain", "return kind == ORACLE_D4 ? 2.0 : 1.0;", "return kind == ORACLE_D4 ? 1.0 : 1.0;"),
    ("MS transposed into LL", "Y[i * W + j] = gain * ms[b][i * W2 + j];", "Y[i * W + j] = gain * ms[b][j * W2 + i];"),
    ("adjoint drops the gain", "grad_ms[b][i * W2 + j] = gain * Y[i * W + j];",
     "grad_ms[b][i * W2 + j] = Y[i * W + j];"),
    ("adjoint keeps the LL", "                Y[i * W + j] = 0.0;\n", "                Y[i * W + j] *= 1.0;\n"),
    ("uint8 rounds half up", "y[k] = (uint8_t)nearbyint(v);", "y[k] = (uint8_t)floor(v + 0.5);"),
    ("ERGAS drops d_h/d_l", "return 100.0 * 0.5 * sqrt(acc / (double)B);", "return 100.0 * sqrt(acc / (double)B);"),
    ("ERGAS reference transposed", "img_at(ms[b], mtype, (y / 2) * W2 + x / 2)", "img_at(ms[b], mtype, (x / 2) * W2 + y / 2)"),
    ("Q numerator factor", "return 4.0 * cxy * mx * my / den;", "return 2.0 * cxy * mx * my / den;"),
    ("Q degenerate window", "if (den == 0.0) return same ? 1.0 : 0.0;", "if (den == 0.0) return 1.0;"),
    ("Q sample variance", "    vx /= n;\n", "    vx /= n - 1.0;\n"),
    ("D_lambda normalisation", "dl /= (double)(B * (B - 1));", "dl /= (double)(B * B);"),
    ("PAN~ block mean", "                 img_at(pan, ptype, (2 * i + 1) * W + 2 * j + 1)) /\n                4.0;",
     "                 img_at(pan, ptype, (2 * i + 1) * W + 2 * j + 1)) /\n                2.0;"),
    ("QNR product", "*qnr = (1.0 - dl) * (1.0 - ds);", "*qnr = (1.0 - dl) + (1.0 - ds) - 1.0;"),
    ("point evaluator: LL swap bounds", "if (i < c->H / 2 && k < c->W / 2) return c->gain * ms_at(c, i, k);",
     "if (i < c->H / 2 && k <= c->W / 2) return c->gain * ms_at(c, i, k);"),
    ("point evaluator: row pass length", "const int nt = inv1d_taps(c->w, c->W, x, idx, wt);",
     "const int nt = inv1d_taps(c->w, c->H, x, idx, wt);"),
    ("point dwt2: column taps", "const int nt = fwd1d_taps(c.w, H, is[k], idx, wt);",
     "const int nt = fwd1d_taps(c.w, W, is[k], idx, wt);"),
    ("MS read transposed (point evaluator)", "return c->ms ? c->ms[i * W2 + j] : (double)c->ms_u8[i * W2 + j];",
     "return c->ms ? c->ms[j * W2 + i] : (double)c->ms_u8[i * W2 + j];"),
    ("point adjoint: LL zeroing bounds", "if (i < c->H / 2 && k < c->W / 2) return 0.0;",
     "if (i < c->H / 2 && k <= c->W / 2) return 0.0;"),
    ("point adjoint: forward users miss a neighbour", "for (long d = -2; d <= 1; ++d) {",
     "for (long d = 0; d <= 1; ++d) {"),
    ("point adjoint: inverse users miss the next pair", "for (long d = -2; d <= 5; ++d) cand",
     "for (long d = -2; d <= 1; ++d) cand"),
    ("point adjoint: grad MS without the gain", "out_ms[(long)b * nm + k] = gain * adj_col_inv(",
     "out_ms[(long)b * nm + k] = adj_col_inv("),
    ("point adjoint: window row offset sign", "const long r = ((y - c->gy0) % c->H + c->H) % c->H;",
     "const long r = ((y + c->gy0) % c->H + c->H) % c->H;"),
    ("point adjoint: column pass over the row length", "const int nu = users1d(1, c->w, c->H, i, o, wt);",
     "const int nu = users1d(1, c->w, c->W, i, o, wt);"),
]


def _build(src_text: str, out_dir: str, tag: int) -> str:
    c = os.path.join(out_dir, f"mutant{tag}.c")
    so = os.path.join(out_dir, f"mutant{tag}.so")
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O1", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-o", so, c, "-lm"],
                   check=True, capture_output=True)
    return so


def test_every_mutant_is_unique_text():
    src = open(SRC).read()
    for name, old, new in MUTANTS:
        assert src.count(old) == 1, name
        assert old != new, name


def test_pins_catch_every_planted_mistake():
    pytest.importorskip("numpy")
    src = open(SRC).read()
    with tempfile.TemporaryDirectory() as tmp:
        procs = []
        for k, (name, old, new) in enumerate(MUTANTS):
            so = _build(src.replace(old, new, 1), tmp, k)
            env = dict(os.environ, DWTFUSE_ORACLE_LIB=so, OMP_NUM_THREADS="1")
            cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                   os.path.join(ROOT, "tests", "test_oracle_pins.py")]
            procs.append((name, subprocess.Popen(cmd, cwd=ROOT, env=env, stdout=subprocess.PIPE,
                                                 stderr=subprocess.STDOUT)))
        survivors = []
        for name, p in procs:
            p.communicate(timeout=600)
            if p.returncode == 0:
                survivors.append(name)
        assert not survivors, f"pins did not catch: {survivors}"
