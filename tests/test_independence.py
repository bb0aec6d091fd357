"""The oracle and the CUDA path share no code, and the product never routes
through the oracle: the oracle's sources include and import nothing of the
package, the package's sources (Python and CUDA/C++) never name the oracle,
and only the seeded input module (which holds no method arithmetic) is
imported by both sides' tests."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _files(patterns):
    out = []
    for p in patterns:
        out += glob.glob(os.path.join(ROOT, p), recursive=True)
    return sorted(out)


def test_oracle_uses_nothing_of_the_package():
    for f in _files(["oracle/*.py", "oracle/*.cpp", "oracle/*.h"]):
        text = open(f).read()
        assert "paper_1411_4622_gb300" not in text, f
        for inc in re.findall(r'#include\s+"([^"]+)"', text):
            assert os.path.dirname(inc) == "" and os.path.exists(os.path.join(ROOT, "oracle", inc)), (f, inc)


def test_package_never_names_the_oracle():
    for f in _files(["paper_1411_4622_gb300/*.py", "paper_1411_4622_gb300/csrc/*", "include/*.h"]):
        text = open(f, errors="replace").read()
        code = re.sub(r"#.*|//.*|/\*.*?\*/|\"\"\".*?\"\"\"", "", text, flags=re.S)
        assert not re.search(r"\bimport\s+oracle\b|\bfrom\s+oracle\b|liboracle|oracle/", code), f


def test_seeded_inputs_hold_no_method_arithmetic():
    """synth.py (shared by both sides' tests) imports only numpy and the
    standard library and defines input generators and error measures only:
    no table, projection, cost, annealing or SIRT step."""
    text = open(os.path.join(ROOT, "paper_1411_4622_gb300", "synth.py")).read()
    text = re.sub(r'""".*?"""', "", text, flags=re.S)
    imports = set(re.findall(r"^(?:from|import)\s+([\w.]+)", text, flags=re.M))
    assert imports <= {"__future__", "math", "dataclasses", "numpy"}, imports
    defs = set(re.findall(r"^def\s+(\w+)", text, flags=re.M))
    assert defs <= {"bins_for", "angles_for", "random_ellipses", "rasterize", "phantom", "disk_mask",
                    "initial_image", "gaussian_noise", "poisson_noise", "rmse", "nrmse", "slice_seeds"}, defs
