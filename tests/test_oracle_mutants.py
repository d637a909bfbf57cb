"""The oracle's pins must reject an oracle with a planted mistake.

Each case copies veckm_oracle.c, plants one plausible mistake (a wrong sign,
a swapped axis, a dropped normaliser, a wrong window bound, a wrong output
row), compiles the copy on the CPU and reruns the pins of
test_oracle_pins.py against it.  At least one pin has to fail for every
mutant; otherwise the pins would not be evidence of anything.
"""
import inspect
import subprocess

import pytest

import oracle
from tests import test_oracle_pins as pins

MUTANTS = {
    "conjugate_sign": ("ci = -sin(ut * T[d]);", "ci = sin(ut * T[d]);"),
    "spatial_axes_swapped": ("const double *yr = sy_re + (b + dy) * D, *yi = sy_im + (b + dy) * D;",
                             "const double *yr = sx_re + (b + dy) * D, *yi = sx_im + (b + dy) * D;"),
    "no_normaliser": ("re[d] = vr / (double)cnt;", "re[d] = vr;"),
    "direct_x_sign": ("const double ux = dx > 0 ? (double)ex / dx : 0.0;",
                      "const double ux = dx > 0 ? -(double)ex / dx : 0.0;"),
    "window_uses_dy_for_x": ("if (ex < -dx || ex > dx || ey < -dy || ey > dy) continue;",
                             "if (ex < -dy || ex > dy || ey < -dy || ey > dy) continue;"),
    "pooled_window_off_by_one": ("for (int32_t a = -dx; a <= dx; ++a) {\n            const int32_t px",
                                 "for (int32_t a = -dx; a < dx; ++a) {\n            const int32_t px"),
    "spatial_product_sign": ("const double sr = xr[d] * yr[d] - xi[d] * yi[d];",
                             "const double sr = xr[d] * yr[d] + xi[d] * yi[d];"),
    "mlp_second_row": ("o1 += (double)W2[hidden + h] * a;", "o1 += (double)W2[h] * a;"),
    "mlp_no_relu": ("if (a < 0.0) a = 0.0;", "if (a < -1e300) a = 0.0;"),
    "mlp_bias_dropped": ("double a = (double)b1[h];", "double a = 0.0;"),
    "kde_conjugate": ("s += emb[d] * cos(a) + emb[D + d] * sin(a);",
                      "s += emb[d] * cos(a) - emb[D + d] * sin(a);"),
    "time_origin_ignored": ("const double ut = (double)((int64_t)t[k] - (int64_t)t_ref) / dt_us;\n        double *r",
                            "const double ut = (double)((int64_t)t[k]) / dt_us * 1.0000001;\n        double *r"),
}


def _pin_calls():
    """Every pin, with the first parameter set of each parametrized one."""
    calls = []
    for name, fn in inspect.getmembers(pins, inspect.isfunction):
        if not name.startswith("test_"):
            continue
        marks = getattr(fn, "pytestmark", [])
        kwargs_list = [{}]
        for m in marks:
            if m.name == "parametrize":
                argnames = [a.strip() for a in m.args[0].split(",")] if isinstance(m.args[0], str) else m.args[0]
                new = []
                for kw in kwargs_list:
                    for vals in m.args[1]:
                        vals = vals if len(argnames) > 1 else (vals,)
                        new.append({**kw, **dict(zip(argnames, vals))})
                kwargs_list = new
        for kw in kwargs_list:
            calls.append((name, fn, kw))
    return calls


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_reject_mutant(mutant, tmp_path):
    src = open(oracle.SOURCE).read()
    a, b = MUTANTS[mutant]
    assert src.count(a) == 1, f"mutation site for {mutant} not found exactly once"
    path = tmp_path / "mut.c"
    path.write_text(src.replace(a, b))
    lib = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", str(lib), str(path), "-lm"],
                   check=True)
    failed = []
    with oracle.using_library(str(lib)):
        for name, fn, kw in _pin_calls():
            try:
                if "tmp_path" in inspect.signature(fn).parameters:
                    kw = {**kw, "tmp_path": tmp_path}
                fn(**kw)
            except (AssertionError, oracle.OracleError):
                failed.append(name)
    assert failed, f"no pin rejects the mutant {mutant}"
