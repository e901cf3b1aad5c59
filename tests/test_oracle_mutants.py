"""Mutation tests of the oracle's Python functions (Alg. 1's rules, the padded
window, the two-stage search, NMI, SWMI, volumes): plant one plausible mistake
in a copy of the oracle source and check that at least one pin fails.  The C
direct method has its own mutants in test_oracle.py.

Each mutant runs in a child process that re-executes the mutated source in the
oracle module's namespace (so the C library and paths stay those of the real
oracle), then runs the pins.  A pin failure or any exception counts as caught;
the unmutated control must pass every pin."""
import os
import subprocess
import sys

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

_MUTATIONS = {
    "gate_strict": ("ok = n.astype(np.float64) >= thr", "ok = n.astype(np.float64) > thr"),
    "align_not_strict": ("        if i_t > best[2]:", "        if i_t >= best[2]:"),
    "window_drops_last_row": ("rows = np.arange(H_B - Hp, 1) + Hp - 1", "rows = np.arange(H_B - Hp, 0) + Hp - 1"),
    "refine_not_strict": ("""        if mi > best[4]:
            best, theta_best = (n_grid + i, dy, dx, n, mi), th""", """        if mi >= best[4]:
            best, theta_best = (n_grid + i, dy, dx, n, mi), th"""),
    "refine_half_width": ("th = base + (2.0 * float(u) - 1.0) * 2.0 * np.pi / n_grid",
                          "th = base + (2.0 * float(u) - 1.0) * np.pi / n_grid"),
    "nmi_halved": ("out[ok] = (ha[ok] + hb[ok]) / hab[ok]", "out[ok] = (ha[ok] + hb[ok]) / (2.0 * hab[ok])"),
    "swmi_one_weight": ("w = wa[ya0:ya1, xa0:xa1] * wb[ya0 + dy:ya1 + dy, xa0 + dx:xa1 + dx]",
                        "w = wb[ya0 + dy:ya1 + dy, xa0 + dx:xa1 + dx]"),
    "swmi_natural_log": ("mi[r, c] = float((p[nz] * np.log2(p[nz] / (pa @ pb)[nz])).sum())",
                         "mi[r, c] = float((p[nz] * np.log(p[nz] / (pa @ pb)[nz])).sum())"),
    "cmif3_depth_shift_dropped": ("b = B[z0 + dz:z1 + dz, y0 + dy:y1 + dy, x0 + dx:x1 + dx]",
                                  "b = B[z0:z1, y0 + dy:y1 + dy, x0 + dx:x1 + dx]"),
    "cmif3_nmi_inverted": ("nmi_map[zi * R2 + r, c] = (entropy(pa.ravel()) + entropy(pb.ravel())) / h_ab",
                           "nmi_map[zi * R2 + r, c] = h_ab / (entropy(pa.ravel()) + entropy(pb.ravel()))"),
}

_RUN_PINS = r"""
import sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import oracle
src = open(oracle.__file__).read()
old, new = {old!r}, {new!r}
if old:
    src = src.replace(old, new)
exec(compile(src, oracle.__file__, "exec"), oracle.__dict__)
import test_oracle as t1, test_oracle_alg1 as t2
pins = [t1.test_gamma_argmax_and_align_rules, t1.test_planted_shift_recovered,
        t2.test_template_cut_out_of_reference, t2.test_two_stage_rules, t2.test_nmi_closed_forms,
        t2.test_swmi_pins, t2.test_cmif3_pins]
pins += [lambda: t2.test_padded_window_equals_unpadded_cmif(((13, 11), (7, 6)), 0.3),
         lambda: t2.test_padded_equals_gated_full_map_for_full_masks(0.5)]
failed = []
for pin in pins:
    try:
        pin()
    except Exception as e:
        failed.append(type(e).__name__)
print(failed)
sys.exit(3 if failed else 0)
"""


def _run(old, new):
    code = _RUN_PINS.format(root=ROOT, tests=HERE, old=old, new=new)
    return subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)


def test_control_passes_every_pin():
    r = _run("", "")
    assert r.returncode == 0, r.stdout + r.stderr


@pytest.mark.parametrize("name", sorted(_MUTATIONS))
def test_python_oracle_mutants_are_caught(name):
    old, new = _MUTATIONS[name]
    assert open(oracle.__file__).read().count(old) == 1, f"mutation {name} does not apply"
    r = _run(old, new)
    assert r.returncode != 0, f"mutation {name} was not caught by any pin"
