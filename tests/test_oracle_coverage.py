"""Every public function of the oracle is exercised by a pin test (the
`-m "not gpu"` tests that check the oracle against closed forms, invariants,
brute force or the paper's printed values), so none is left unpinned."""
import ast
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# pin tests: the oracle's own tests plus the host tests that hold it to the
# paper's printed parameters and to an independent library solve
PIN_FILES = glob.glob(os.path.join(ROOT, "tests", "test_oracle_*.py")) + [
    os.path.join(ROOT, "tests", "test_paper_system.py"), os.path.join(ROOT, "tests", "test_bench_cufft.py")]
INFRA = {"build", "lib"}


def test_every_oracle_function_is_pinned():
    tree = ast.parse(open(os.path.join(ROOT, "oracle", "__init__.py")).read())
    funcs = [n.name for n in tree.body if isinstance(n, ast.FunctionDef) and not n.name.startswith("_")]
    src = "".join(open(f).read() for f in PIN_FILES if os.path.basename(f) != "test_oracle_coverage.py")
    missing = [f for f in funcs if f not in INFRA and not re.search(r"\b(O|oracle_lib)\." + f + r"\b", src)]
    assert funcs and not missing, missing
