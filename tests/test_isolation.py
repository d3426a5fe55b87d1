"""The product package never imports the oracle (which is test infrastructure),
and the oracle never imports the product package: the two share only the
seeded input generators (paper_2403_11166_gb300/inputs.py)."""
import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _imports(path):
    tree = ast.parse(open(path).read(), path)
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name
        elif isinstance(node, ast.ImportFrom):
            yield (node.module or "") if node.level == 0 else "." * node.level + (node.module or "")


def _py_files(d):
    for base, _, files in os.walk(os.path.join(ROOT, d)):
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(base, f)


def test_package_does_not_import_the_oracle():
    for path in _py_files("paper_2403_11166_gb300"):
        for mod in _imports(path):
            assert not mod.split(".")[0] == "oracle", (path, mod)


def test_oracle_does_not_import_the_package():
    for path in _py_files("oracle"):
        for mod in _imports(path):
            assert not mod.startswith("paper_2403_11166_gb300"), (path, mod)
