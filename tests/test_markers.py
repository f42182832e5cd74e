"""The test modules that need a GPU are marked so that `-m gpu` selects them
and `-m "not gpu"` leaves them out: every tests/test_gpu_*.py module (and the
allocation-free test, which runs last) sets the module-wide gpu mark, and no
other module does."""

import ast
import os

HERE = os.path.dirname(os.path.abspath(__file__))
GPU_MODULES_BY_NAME = ("test_zz_no_alloc.py",)


def _module_marks(path):
    tree = ast.parse(open(path).read())
    for node in tree.body:
        if isinstance(node, ast.Assign) and any(isinstance(t, ast.Name) and t.id == "pytestmark" for t in node.targets):
            return ast.unparse(node.value)
    return ""


def test_gpu_modules_are_marked():
    for name in sorted(os.listdir(HERE)):
        if not (name.startswith("test_") and name.endswith(".py")):
            continue
        marks = _module_marks(os.path.join(HERE, name))
        if name.startswith("test_gpu_") or name in GPU_MODULES_BY_NAME:
            assert "pytest.mark.gpu" in marks, name
        else:
            assert "pytest.mark.gpu" not in marks, name
