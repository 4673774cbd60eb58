"""Planted mistakes in the oracle must be caught by its pins.

Each case copies ``oracle/oracle.c``, makes one textual change of the kind a
careless transcription of the paper's definitions would make (a flipped sign,
a dropped term or factor, a wrong index, a transposed operand), compiles the
copy on the CPU and runs every pin on it in a child process.  At least one
pin has to fail (a mutant that crashes the child counts as caught).
"""
import json
import os
import subprocess
import sys

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))

_RUNNER = """
import json, sys
sys.path[:0] = [{here!r}, {root!r}]
import oracle
from oracle_pins import ALL_PINS
lib = oracle.load({so!r})
failed = []
for pin in ALL_PINS:
    try:
        pin(lib)
    except Exception as e:
        failed.append(pin.__name__)
print(json.dumps(failed))
"""

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    # Eq. 1 / Eq. 2 sign of the exponent
    "root_sign": ("t[p] = cos(a) + (double)sign * I * sin(a);",
                  "t[p] = cos(a) - (double)sign * I * sin(a);"),
    # Cooley-Tukey combine: twiddle index loses its s*m term
    "combine_index": ("roots[((q * (k + s * m)) % n) * step] * y[q * m + k]",
                      "roots[((q * k) % n) * step] * y[q * m + k]"),
    # direct DFT uses j+k instead of j*k
    "direct_index": ("acc += x[j * stride] * roots[((j * k) % n) * step];",
                     "acc += x[j * stride] * roots[((j + k) % n) * step];"),
    # normalisation step of the inverse dropped
    "no_normalisation": ("f[l * n2 + i] = creal(out[i]) * scale;",
                         "f[l * n2 + i] = creal(out[i]);"),
    # Hermitian extension off by one
    "hermitian_index": ("line[k] = (k <= n2 / 2) ? y[k] : conj(y[n2 - k]);",
                        "line[k] = (k <= n2 / 2) ? y[k] : conj(y[n2 - k - 1]);"),
    # Hermitian extension without the conjugate
    "hermitian_conj": ("line[k] = (k <= n2 / 2) ? y[k] : conj(y[n2 - k]);",
                       "line[k] = (k <= n2 / 2) ? y[k] : y[n2 - k];"),
    # Nyquist entry counted twice on the halved axis
    "nyquist_doubled": ("if (n2 % 2 == 0) line[n2 / 2] = creal(y[n2 / 2]);",
                        "if (n2 % 2 == 0) line[n2 / 2] = 2.0 * creal(y[n2 / 2]);"),
    # axis-1 pass run with the axis-0 length (transposed operand)
    "axis_length_swap": ("if (c2c_axis(F, n1, n0 * m1, m1, n1 * m1, m1, -1)) return -1;",
                         "if (c2c_axis(F, n0, n0 * m1, m1, n1 * m1, m1, -1)) return -1;"),
    # inverse run with the forward sign on axis 0
    "inverse_sign": ("if (c2c_axis(work, n0, n1 * m1, n1 * m1, 0, n1 * m1, +1) ||",
                     "if (c2c_axis(work, n0, n1 * m1, n1 * m1, 0, n1 * m1, -1) ||"),
    # half spectrum one entry short
    "half_length": ("long m1 = n2 / 2 + 1;\n    long lines = n0 * n1;\n    cplx *roots = root_table(n2, -1);",
                    "long m1 = n2 / 2 + 1;\n    long lines = n0 * n1;\n    cplx *roots = root_table(n2, -1);\n    m1 -= (n2 > 4);"),
    # adjoint of the inverse: doubling weight on the wrong planes
    "adjoint_weights": ("G[l * m1 + k] *= (edge ? 1.0 : 2.0) * scale;",
                        "G[l * m1 + k] *= (edge ? 2.0 : 1.0) * scale;"),
    # adjoint of the forward with the forward sign
    "adjoint_sign": ("if (c2c_axis(full, n2, n0 * n1, 1, n2, 1, +1) ||",
                     "if (c2c_axis(full, n2, n0 * n1, 1, n2, 1, -1) ||"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    so = oracle.build(str(path), str(tmp_path / "libmutant.so"))
    code = _RUNNER.format(here=HERE, root=os.path.dirname(HERE), so=so)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                       timeout=300, env={**os.environ, "OMP_NUM_THREADS": "2"})
    if r.returncode != 0:
        return  # the mutant crashed under the pins: caught
    failed = json.loads(r.stdout.strip().splitlines()[-1])
    assert failed, f"no pin caught mutant {name}"
