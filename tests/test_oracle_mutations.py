"""The oracle's pins must catch plausible mistakes: each case plants one mistake in a copy of the
oracle's C source (on the CPU), rebuilds it and checks that the pin suite now fails."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = {
    "p_agg of the child instead of the node": (
        "double pagg = p_in(t, T, a, sampling);\n                    prr",
        "double pagg = p_in(t, c, a, sampling);\n                    prr"),
    "swap with the wrong sign": ("return s - node_term(t, k, v, q);", "return node_term(t, k, v, q) - s;"),
    "roulette threshold at the node's cell size": (
        "float X = ldexpf(dv > bv ? dv : bv, -(t->bits / 3) * (t->level[c] - t->level[v]));",
        "float X = dv > bv ? dv : bv;"),
    "roulette continues when the draw is above p": ("if (!((double)u * (double)dc < (double)X)) return 0;",
                                                    "if ((double)u * (double)dc < (double)X) return 0;"),
    "p(K >= k) missing the current step": (
        "prr *= (double)p;\n                    Fa += delta / (pagg * prr);",
        "Fa += delta / (pagg * prr);\n                    prr *= (double)p;"),
    "centre of mass not divided by the mass": ("t->com[3 * v + a] = s[a] / m;", "t->com[3 * v + a] = s[a];"),
    "unnormalised child prefix": ("(float)(pre / tot);", "(float)(pre);"),
    "one random word for both draws": ("int64_t c = pick_child(t, T, x[0], sampling);",
                                       "int64_t c = pick_child(t, T, x[1], sampling);"),
    "winding orientation": ("return (dx * dip[0] + dy * dip[1] + dz * dip[2]) / (4.0 * M_PI * r2 * r);",
                            "return -(dx * dip[0] + dy * dip[1] + dz * dip[2]) / (4.0 * M_PI * r2 * r);"),
    "Morton interleave y before x": (
        "((uint64_t)((cx >> b) & 1u) << 2) | ((uint64_t)((cy >> b) & 1u) << 1) |",
        "((uint64_t)((cy >> b) & 1u) << 2) | ((uint64_t)((cx >> b) & 1u) << 1) |"),
    "single-child chains kept": (
        "if (runs == 1 && t->collapse) { x->level += 1; continue; }",
        "if (runs == 1 && !t->collapse) { x->level += 1; continue; }"),
    "tight box without the zero-extent rule": ("if (b == 0.0 && box_mode == 1) b = ldexp(",
                                               "if (b == 0.0 && box_mode == 3) b = ldexp("),
    "tight box radius for its diameter": ("double b = sqrt(s2);", "double b = 0.5 * sqrt(s2);"),
    "subdomains one generation too deep": (
        "if (gen[v] == sub_gen || (gen[v] < sub_gen && t->nchild[v] == 0))",
        "if (gen[v] == sub_gen + 1 || (gen[v] < sub_gen + 1 && t->nchild[v] == 0))"),
    "Barnes-Hut cut without its leaves": (
        "if (t->nchild[v] == 0 || ffratio32(t, v, q32) >= beta) { out[(*n)++] = v; return; }",
        "if (t->nchild[v] == 0) return;\n    if (ffratio32(t, v, q32) >= beta) { out[(*n)++] = v; return; }"),
    "odd depths reuse the even depth's words": ("w[0] = x[2 * (k & 1u)];\n    w[1] = x[2 * (k & 1u) + 1];",
                                                "w[0] = x[0];\n    w[1] = x[1];"),
    "Philox key schedule": ("if (round > 0) { k0 += weyl0; k1 += weyl1; }",
                            "if (round > 1) { k0 += weyl0; k1 += weyl1; }"),
    "winding gradient missing its r^-5 term": (
        "for (int a = 0; a < 3; ++a) g[a] = (-dip[a] / r3 + 3.0 * dn * d[a] / r5) / (4.0 * M_PI);",
        "for (int a = 0; a < 3; ++a) g[a] = (-dip[a] / r3) / (4.0 * M_PI);"),
    "Coulomb gradient sign": ("for (int a = 0; a < 3; ++a) g[a] = c * d[a];\n        return;\n    }\n    case K_WINDING",
                              "for (int a = 0; a < 3; ++a) g[a] = -c * d[a];\n        return;\n    }\n    case K_WINDING"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(tmp_path, name):
    src, dst = MUTATIONS[name]
    for d in ("oracle", "tests", "paper_2506_02219_gb300"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d,
                        ignore=shutil.ignore_patterns("*.so", "_build", "__pycache__", "test_oracle_mutations.py"))
    c = tmp_path / "oracle" / "sbh_oracle.c"
    text = c.read_text()
    assert src in text, "mutation anchor not found"
    c.write_text(text.replace(src, dst, 1))
    tests = [f"tests/{f}" for f in ("test_oracle_philox.py", "test_oracle_brute.py", "test_oracle_tree.py",
                                    "test_oracle_estimator.py", "test_oracle_grad.py", "test_oracle_readings.py")]
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *tests],
                       cwd=tmp_path, capture_output=True, text=True, timeout=900)
    assert r.returncode == 1, f"pins did not catch: {name}\n{r.stdout[-2000:]}"
