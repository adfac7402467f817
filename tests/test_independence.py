"""The product path and the oracle are independent: nothing in the package (Python binding, CUDA sources,
headers) imports, includes or names a file of ``oracle/``, the oracle imports nothing of the package, and
the shared input generators in ``phantoms/`` import neither."""
import ast
import os
import re

PACKAGE = "paper_1910_13844_gb300"


def _py_imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            mods.add(node.module.split(".")[0])
    return mods


def _files(root, exts):
    for dirpath, _, names in os.walk(root):
        if "__pycache__" in dirpath or "_build" in dirpath:
            continue
        for n in names:
            if n.endswith(exts):
                yield os.path.join(dirpath, n)


def test_package_never_imports_the_oracle(repo_root):
    for path in _files(os.path.join(repo_root, PACKAGE), (".py",)):
        assert "oracle" not in _py_imports(path), path


def test_cuda_sources_include_nothing_from_the_oracle(repo_root):
    roots = [os.path.join(repo_root, PACKAGE, "csrc"), os.path.join(repo_root, "include")]
    for root in roots:
        for path in _files(root, (".cu", ".cuh", ".h", ".cpp")):
            for inc in re.findall(r'#\s*include\s*[<"]([^>"]+)[>"]', open(path).read()):
                assert "oracle" not in inc, (path, inc)


def test_oracle_and_input_generators_import_nothing_of_the_package(repo_root):
    for sub in ("oracle", "phantoms"):
        for path in _files(os.path.join(repo_root, sub), (".py",)):
            mods = _py_imports(path)
            assert PACKAGE not in mods, path
            if sub == "phantoms":
                assert "oracle" not in mods, path
