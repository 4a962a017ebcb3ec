"""The oracle and the CUDA path stay apart (no GPU needed): no module of the
package names the oracle, the two share no header, table or helper (each
includes only its own files and the system's), bench.py reaches the oracle
only in its CPU-baseline leg, and the oracle declares itself test
infrastructure.  The seeded-input module is the one thing both sides take,
and it holds no step of the method (no collision, event or field update)."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1704_01202_gb300")
CSRC = os.path.join(PKG, "csrc")
ORACLE = os.path.join(ROOT, "oracle")


def _files(d, exts):
    for base, _, names in os.walk(d):
        if "_build" in base or "__pycache__" in base:
            continue
        for n in names:
            if n.endswith(exts):
                yield os.path.join(base, n)


def _py_imports(path):
    t = ast.parse(open(path).read())
    out = set()
    for node in ast.walk(t):
        if isinstance(node, ast.Import):
            out.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            out.add(node.module.split(".")[0])
    return out


def test_package_never_reaches_the_oracle():
    for f in _files(PKG, (".py",)):
        assert "oracle" not in _py_imports(f), f
    for f in _files(PKG, (".py", ".cu", ".cuh", ".h")):
        src = open(f).read()
        assert "liboracle" not in src and "oracle.h" not in src and "orc_" not in src, f


def test_no_shared_sources():
    """Each side includes only its own files and system headers."""
    for f in _files(CSRC, (".cu", ".cuh")):
        for inc in re.findall(r'#include\s*"([^"]+)"', open(f).read()):
            assert os.path.exists(os.path.join(CSRC, inc)), (f, inc)
            assert "oracle" not in inc
    for f in _files(ORACLE, (".c", ".h")):
        for inc in re.findall(r'#include\s*"([^"]+)"', open(f).read()):
            assert os.path.exists(os.path.join(ORACLE, inc)), (f, inc)
            assert not inc.startswith("pic"), (f, inc)
    for f in _files(ORACLE, (".py",)):
        assert "paper_1704_01202_gb300" not in _py_imports(f), f


def test_bench_reaches_the_oracle_only_for_the_cpu_baseline():
    t = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    users = []
    for fn in [n for n in ast.walk(t) if isinstance(n, ast.FunctionDef)]:
        for node in ast.walk(fn):
            if isinstance(node, (ast.Import, ast.ImportFrom)):
                names = [a.name for a in node.names] if isinstance(node, ast.Import) else [node.module]
                if any(n and n.split(".")[0] == "oracle" for n in names):
                    users.append(fn.name)
    module_level = [n for n in t.body if isinstance(n, (ast.Import, ast.ImportFrom))]
    assert not any("oracle" in ast.dump(n) for n in module_level)
    assert users == ["cpu_baseline"], users


def test_oracle_declares_itself_test_infrastructure():
    assert "test infrastructure" in open(os.path.join(ORACLE, "__init__.py")).read().lower()
    assert "TEST INFRASTRUCTURE ONLY" in open(os.path.join(ORACLE, "oracle.c")).read()


def test_input_module_holds_no_step_of_the_method():
    src = open(os.path.join(ROOT, "pic_inputs", "__init__.py")).read()
    for word in ("def collide", "def boris", "def deposit", "def lotz", "def photoionize", "def field_step",
                 "import oracle", "import paper_1704_01202_gb300"):
        assert word not in src, word
