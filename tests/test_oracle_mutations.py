"""Plant plausible mistakes in a copy of the oracle (on the CPU, never the
CUDA path) and check that the pins catch every one of them: a dropped term,
a wrong sign, a wrong index, a transposed operand, a wrong state slot, a
broken cascade hand-off, and broken adjoint terms."""
import os
import shutil
import subprocess

import pytest

import oracle
import pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "sosfilt_oracle.c")

MUTATIONS = [
    ("drop_b2_term", "acc += b2 * in[n - 2] - a2 * out[n - 2];", "acc += - a2 * out[n - 2];"),
    ("sign_a1", "acc += b1 * in[n - 1] - a1 * out[n - 1];", "acc += b1 * in[n - 1] + a1 * out[n - 1];"),
    ("index_b1", "acc += b1 * in[n - 1] - a1 * out[n - 1];", "acc += b1 * in[n - 2] - a1 * out[n - 1];"),
    ("zi_slot_swap", "if (n == 0) acc += zi[0];", "if (n == 0) acc += zi[1];"),
    ("a1_a2_transposed", "c[3] = row[4] / a0;", "c[3] = row[5] / a0;"),
    ("b0_not_normalised", "c[0] = row[0] / a0;", "c[0] = row[0];"),
    ("zf_z2_wrong_b", "z2 += b2 * in[T - 1] - a2 * out[T - 1];", "z2 += b1 * in[T - 1] - a2 * out[T - 1];"),
    ("zf_len1_state", "if (T == 1) z1 += zi[1];", "if (T == 1) z1 += zi[0];"),
    ("cascade_handoff", "((K[c] - 1 - k) % 2 == 0) ? dst : buf", "((K[c] - k) % 2 == 0) ? dst : buf"),
    ("zi_section_index", "const double *z0 = zi ? zi + ((int64_t)c * kmax + k) * 2 : zero2;\n            double zfk[2];\n            double *out",
     "const double *z0 = zi ? zi + ((int64_t)c * kmax) * 2 : zero2;\n            double zfk[2];\n            double *out"),
    ("adjoint_drop_a2_feedback", "            g_out[n - 2] -= g * a2;\n", "\n"),
    ("adjoint_a0_sign", "gr[3] = -(gc[0]", "gr[3] = (gc[0]"),
    ("adjoint_b1_index", "g_in[n - 1] += g * b1;", "g_in[n - 2 >= 0 ? n - 2 : 0] += g * b1;"),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_mutation(tmp_path, name, old, new):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {name}"
    mutant = src.replace(old, new, 1)
    cpath = tmp_path / "mutant.c"
    cpath.write_text(mutant)
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O1", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", str(lib),
                    str(cpath)], check=True)
    orc = oracle.Oracle(str(lib))
    caught = []
    for pin in pins.ALL_PINS:
        try:
            pin(orc)
        except ImportError:
            continue
        except Exception:  # noqa: BLE001 - any failure counts as detection
            caught.append(pin.__name__)
    assert caught, f"mutation {name} slipped past every pin"
