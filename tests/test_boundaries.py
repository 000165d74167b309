"""The oracle and the CUDA product path are independent. The product package neither imports nor
loads anything under oracle/. The oracle imports nothing from the product package, and its C
source includes no product header. The only module both sides may take inputs from,
paper_1904_03057_gb300/inputs.py, holds no method arithmetic: it does not import the binding or
the API."""
import ast
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1904_03057_gb300")


def _imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            mod = ("." * node.level) + (node.module or "")
            names.add(mod)
            names.update(f"{mod}.{a.name}" for a in node.names)
    return names


def test_product_package_does_not_touch_the_oracle():
    for path in glob.glob(os.path.join(PKG, "*.py")):
        assert not any(n == "oracle" or n.startswith("oracle.") for n in _imports(path)), path
        assert "bsk_oracle" not in open(path).read(), path
    for path in glob.glob(os.path.join(PKG, "csrc", "*")):
        text = open(path, errors="replace").read()
        assert not re.search(r'#include\s+"[^"]*oracle', text), path
        assert "orc_" not in text, path


def test_oracle_does_not_touch_the_product():
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        assert not any("paper_1904_03057_gb300" in n or n.startswith(".paper") for n in _imports(path)), path
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.c")) + glob.glob(os.path.join(ROOT, "oracle", "*.h")):
        text = open(path).read()
        includes = re.findall(r'#include\s+[<"]([^>"]+)[>"]', text)
        assert all(not inc.startswith(("bsk", "csrc", "paper_")) for inc in includes), (path, includes)


def test_shared_input_module_holds_no_method():
    names = _imports(os.path.join(PKG, "inputs.py"))
    assert not any(n.endswith(("api", "_native", "learned")) or "oracle" in n for n in names), names
