"""The product path and the oracle stay apart: nothing in the package
imports, includes, links or loads anything under oracle/ or _work/, and the
oracle does not reach into the package's CUDA sources.  Only the seeded
graph generators (graphs.py, gen/) serve both sides, and they hold none of
the method's arithmetic."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2009_10035_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _files(top, exts):
    for d, dirs, files in os.walk(top):
        dirs[:] = [x for x in dirs if x not in ("__pycache__", "_build")]
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def _imports(path):
    tree = ast.parse(open(path).read())
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name
        elif isinstance(node, ast.ImportFrom):
            yield ("." * node.level) + (node.module or "")


def test_package_python_never_imports_the_oracle():
    for path in _files(PKG, (".py",)):
        for name in _imports(path):
            assert not re.match(r"(oracle|_work)(\.|$)", name), (path, name)
        text = open(path).read()
        assert not re.search(r"(^|[/'\"])_work([/'\"]|$)", text, re.M), path
        assert not re.search(r"['\"/]oracle[/'\"]", text), path


def test_cuda_sources_include_nothing_from_the_oracle():
    for path in _files(PKG, (".cu", ".cuh", ".h", ".c", ".cpp")):
        for inc in re.findall(r'#\s*include\s*[<"]([^>"]+)[>"]', open(path).read()):
            assert "oracle" not in inc and "_work" not in inc, (path, inc)


def test_build_compiles_only_package_sources():
    from paper_2009_10035_gb300 import build
    for src in build.sources():
        p = os.path.realpath(src)
        assert p.startswith(os.path.realpath(PKG) + os.sep), src


def test_oracle_does_not_reach_into_the_cuda_path():
    for path in _files(ORACLE, (".py", ".c", ".h")):
        text = open(path).read()
        assert "csrc" not in text and not re.search(r"libf2v\.so", text), path
        if path.endswith(".py"):
            for name in _imports(path):
                assert not re.search(r"(^|\.)f2v$|paper_2009_10035_gb300", name), (path, name)
