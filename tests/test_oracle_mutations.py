"""The oracle's pins are strong enough to catch plausible mistakes: each mutation below is
planted in a copy of oracle.c (on the CPU), the copy is compiled and swapped in for the oracle,
and at least one of the pins of test_oracle_pins.py must fail on it.  The real oracle is
restored afterwards and is untouched on disk."""
import ctypes
import importlib.util
import os
import subprocess

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "oracle.c")

# (name, text in oracle.c, replacement): one plausible slip each
MUTATIONS = [
    ("SpMV drops the last entry of each row",
     "    for (int32_t i = 0; i < n_rows; ++i) {\n        double acc = 0.0;\n"
     "        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {",
     "    for (int32_t i = 0; i < n_rows; ++i) {\n        double acc = 0.0;\n"
     "        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1] - 1; ++k) {"),
    ("SpMV gathers x at the row instead of the column",
     "                acc = fma(val[k], x[col_idx[k]], acc);",
     "                acc = fma(val[k], x[i], acc);"),
    ("CG direction update with the wrong sign",
     "double beta = rho_new / rho;", "double beta = -rho_new / rho;"),
    ("CG step length from p.p instead of p.q",
     "double alpha = rho / dot64(n, p, q);", "double alpha = rho / dot64(n, p, p);"),
    ("CG without the Jacobi preconditioner",
     "        for (int32_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i];\n        double rho_new",
     "        for (int32_t i = 0; i < n; ++i) z[i] = r[i];\n        double rho_new"),
    ("Cuthill-McKee visits neighbours by decreasing degree",
     "if (deg[a] != deg[b]) return deg[a] < deg[b];",
     "if (deg[a] != deg[b]) return deg[a] > deg[b];"),
    ("sliced ELLPACK pads with column 0",
     "sell_col[at] = -1;", "sell_col[at] = 0;"),
    ("column range one short at the top",
     "if (!any || c + 1 > hi) hi = c + 1;", "if (!any || c > hi) hi = c;"),
    ("refinement update of x without the residual's scale",
     "x[i] = x[i] + s * (double)d[i];", "x[i] = x[i] + (double)d[i];"),
    ("adaptive inner tolerance with ||r|| / ||b|| instead of ||b|| / ||r||",
     "double need = 0.5 * rtol * bnorm / rnorm;", "double need = 0.5 * rtol * rnorm / bnorm;"),
    ("adaptive inner tolerance capped with max instead of min",
     "if (need > tol_in) tol_in = need < 0.5 ? need : 0.5;",
     "if (need > tol_in) tol_in = need > 0.5 ? need : 0.5;"),
]


def _pins():
    spec = importlib.util.spec_from_file_location("oracle_pins",
                                                  os.path.join(HERE, "test_oracle_pins.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    out = []
    for name in dir(mod):
        fn = getattr(mod, name)
        if not name.startswith("test_") or not callable(fn):
            continue
        if fn.__code__.co_varnames[:1] != ("oracle",):
            continue
        params = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
        combos = [{}]
        for m in params:
            names = [a.strip() for a in m.args[0].split(",")]
            new = []
            for c in combos:
                for v in m.args[1]:
                    vals = v if len(names) > 1 else (v,)
                    new.append({**c, **dict(zip(names, vals))})
            combos = new
        for kw in combos:
            out.append((name, fn, kw))
    return out


def _load_mutant(path):
    return oracle._configure(ctypes.CDLL(path))


def _failing_pins(lib, pins):
    saved = oracle._lib
    oracle._lib = lib
    failed = []
    try:
        for name, fn, kw in pins:
            try:
                fn(oracle, **kw)
            except Exception:  # an assertion, or the mutant reporting an error
                failed.append(name)
    finally:
        oracle._lib = saved
    return failed


@pytest.mark.parametrize("index", range(len(MUTATIONS)))
def test_pins_catch_planted_mistake(tmp_path, index):
    name, old, new = MUTATIONS[index]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    mutant = tmp_path / "oracle_mutant.c"
    mutant.write_text(src.replace(old, new))
    so = tmp_path / "liboracle_mutant.so"
    subprocess.check_call([os.environ.get("CC", "gcc"), "-O2", "-ffp-contract=off", "-fPIC",
                           "-shared", "-std=c11", "-o", str(so), str(mutant), "-lm"])
    failed = _failing_pins(_load_mutant(str(so)), _pins())
    assert failed, "no pin fails on the mutation: " + name


def test_real_oracle_passes_every_pin():
    assert _failing_pins(oracle.lib(), _pins()) == []
