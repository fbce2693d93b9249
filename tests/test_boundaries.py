"""The oracle and the CUDA path stay apart (CPU): the product package never
imports the oracle, the oracle never imports the product package (inputs
reach it as plain arrays), and the bench runs the oracle only in the
subprocess of its CPU-baseline and reference legs."""
import ast
import glob
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _imports(path):
    tree = ast.parse(open(path).read(), path)
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            out.add(node.module.split(".")[0])
    return out


def test_package_never_imports_the_oracle():
    files = glob.glob(os.path.join(ROOT, "paper_1710_03608_gb300", "**", "*.py"), recursive=True)
    assert files
    for f in files:
        assert "oracle" not in _imports(f), f


def test_cuda_sources_do_not_reference_the_oracle():
    files = glob.glob(os.path.join(ROOT, "paper_1710_03608_gb300", "csrc", "*"))
    files += glob.glob(os.path.join(ROOT, "include", "*.h"))
    assert files
    for f in files:
        assert "oracle" not in open(f).read(), f


def test_oracle_never_imports_the_package():
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        assert "paper_1710_03608_gb300" not in _imports(f), f


def test_bench_runs_the_oracle_only_in_a_subprocess():
    assert "oracle" not in _imports(os.path.join(ROOT, "bench.py"))
