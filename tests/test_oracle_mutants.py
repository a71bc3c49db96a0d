"""The oracle's pins catch planted mistakes.

Each case copies oracle/nef_oracle.c, plants one plausible slip in the copy (a
dropped operand, a wrong exponent, a transposed layout, a mask left out, a
wrong branch of the g-table), builds it on the CPU, and runs the pin suites
(test_oracle_pins.py, test_oracle_lik_pins.py) against that build in a child
process: some pin must fail.  The same is done for the encoder oracle (oracle/mlp.py against
test_mlp_oracle.py).  The committed oracle itself is never modified.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "nef_oracle.c")

MUTANTS = [
    ("contraction drops its first operand",
     "for (int k = 0; k < n_ops; ++k) p *= ops[k][off[k]];",
     "for (int k = 1; k < n_ops; ++k) p *= ops[k][off[k]];"),
    ("a(x, y) with exponent beta instead of beta - 1",
     "*a = powz(x, al) * pow(y, be - 1.0);",
     "*a = powz(x, al) * pow(y, be);"),
    ("b(x, y) with exponent alpha + beta instead of alpha + beta - 1",
     "*b = pow(y, al + be - 1.0);",
     "*b = pow(y, al + be);"),
    ("g-table: the q > 1 branch takes the q < 0 exponent",
     "if (q > 1.0) p = 1.0 - be;",
     "if (q > 1.0) p = al + be - 1.0;"),
    ("update applies g instead of its inverse",
     "return pow(z, 1.0 / p);",
     "return pow(z, p);"),
    ("divergence: sign of the cross term",
     "- powz(x, al) * powz(y, be));",
     "+ powz(x, al) * powz(y, be));"),
    ("factors stored transposed (column-major strides)",
     "for (int p = s->fac_nlet[f] - 1; p >= 0; --p) {",
     "for (int p = 0; p < s->fac_nlet[f]; ++p) {"),
    ("Y stored transposed (column-major strides)",
     "for (int m = s->n_obs - 1; m >= 0; --m) { st[m] = acc; acc *= s->dim[m]; }",
     "for (int m = 0; m < s->n_obs; ++m) { st[m] = acc; acc *= s->dim[m]; }"),
    ("weights ignore the mask",
     "if (mask && !mask[e]) { wa[e] = 0.0; wb[e] = 0.0; continue; }\n        ab_weights(",
     "if (0) { wa[e] = 0.0; wb[e] = 0.0; continue; }\n        ab_weights("),
    ("likelihood weights ignore the mask",
     "if (mask && !mask[e]) { wa[e] = 0.0; wb[e] = 0.0; continue; }\n        lik_ab(",
     "if (0) { wa[e] = 0.0; wb[e] = 0.0; continue; }\n        lik_ab("),
    ("update ignores the epsilon floor",
     "theta[e] = v > eps ? v : eps;",
     "theta[e] = v;"),
    ("negative binomial b(x, y) inverted",
     "*b = (par + x) / (par + y); break;",
     "*b = (par + y) / (par + x); break;"),
    ("binomial b(x, y) without the trial count",
     "*b = n / (1.0 + y); break;",
     "*b = 1.0 / (1.0 + y); break;"),
    ("Jensen-Shannon a(x, y) without the midpoint's 1/2",
     "*a = log((x + y) / (2.0 * y)); *b = 1.0; break;",
     "*a = log((x + y) / y); *b = 1.0; break;"),
    ("Jensen-Shannon update takes g as the identity",
     "static double lik_ginv(int kind, double z) { return kind == 3 ? exp(z) : z; }",
     "static double lik_ginv(int kind, double z) { return z; }"),
]

CHILD = """
import sys
import oracle.core as core
core._SRC = sys.argv[1]
core._LIB_PATH = sys.argv[2]
import pytest
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", "tests/test_oracle_pins.py",
                      "tests/test_oracle_lik_pins.py"]))
"""


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(name, old, new, tmp_path):
    with open(SRC) as fh:
        src = fh.read()
    assert src.count(old) == 1, f"mutation site not unique: {name}"
    mut_src = tmp_path / "nef_oracle.c"
    mut_src.write_text(src.replace(old, new))
    mut_lib = tmp_path / "libnef_oracle_mutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", str(mut_src), "-o", str(mut_lib),
                    "-lm"], check=True)
    r = subprocess.run([sys.executable, "-c", CHILD, str(mut_src), str(mut_lib)], cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"no pin failed for: {name}\n{r.stdout[-2000:]}\n{r.stderr[-2000:]}"


def test_unmutated_copy_passes(tmp_path):
    """Control: the same harness on an unchanged copy passes every pin."""
    mut_src = tmp_path / "nef_oracle.c"
    with open(SRC) as fh:
        mut_src.write_text(fh.read())
    mut_lib = tmp_path / "libnef_oracle_copy.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", str(mut_src), "-o", str(mut_lib),
                    "-lm"], check=True)
    r = subprocess.run([sys.executable, "-c", CHILD, str(mut_src), str(mut_lib)], cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]


MLP_SRC = os.path.join(ROOT, "oracle", "mlp.py")

MLP_MUTANTS = [
    ("softplus derivative taken as 1", "g_z3 = g_out * sigmoid(z3)", "g_z3 = g_out"),
    ("relu derivative of layer 2 dropped", "g_z2 = g_h2 * (z2 > 0.0)", "g_z2 = g_h2"),
    ("square weight gradient transposed", "gW2 = h1.T @ g_z2", "gW2 = g_z2.T @ h1"),
    ("bias gradient averaged instead of summed", "gb1 = g_z1.sum(axis=0)", "gb1 = g_z1.mean(axis=0)"),
    ("loss derivative missing the 1 / (1 + out) factor", "g_out = 2.0 * d / (1.0 + out) / n", "g_out = 2.0 * d / n"),
    ("Adam without bias correction of the second moment", "vh = v / (1.0 - b2 ** t)", "vh = v"),
    ("forward pass skips the second bias", "z2 = h1 @ W2 + b2", "z2 = h1 @ W2"),
]

MLP_CHILD = """
import importlib.util
import sys
import oracle
spec = importlib.util.spec_from_file_location("oracle.mlp", sys.argv[1])
mod = importlib.util.module_from_spec(spec)
spec.loader.exec_module(mod)
sys.modules["oracle.mlp"] = mod
oracle.mlp = mod
import pytest
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", "tests/test_mlp_oracle.py"]))
"""


@pytest.mark.parametrize("name,old,new", MLP_MUTANTS, ids=[m[0] for m in MLP_MUTANTS])
def test_mlp_pins_catch_planted_mistake(name, old, new, tmp_path):
    with open(MLP_SRC) as fh:
        src = fh.read()
    assert src.count(old) == 1, f"mutation site not unique: {name}"
    mut = tmp_path / "mlp.py"
    mut.write_text(src.replace(old, new))
    r = subprocess.run([sys.executable, "-c", MLP_CHILD, str(mut)], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 1, f"no pin failed for: {name}\n{r.stdout[-2000:]}\n{r.stderr[-2000:]}"


def test_mlp_unmutated_copy_passes(tmp_path):
    mut = tmp_path / "mlp.py"
    with open(MLP_SRC) as fh:
        mut.write_text(fh.read())
    r = subprocess.run([sys.executable, "-c", MLP_CHILD, str(mut)], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
