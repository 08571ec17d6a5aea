"""Static checks of bench.py that need no GPU: it parses, and no function binds a local
name that shadows a module-level import (which would make every use of that module in
the function fail before the local binding runs)."""
import ast
import os
import symtable

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _module_imports(tree):
    names = set()
    for node in tree.body:
        if isinstance(node, (ast.Import, ast.ImportFrom)):
            for a in node.names:
                names.add((a.asname or a.name).split(".")[0])
    return names


def _walk(table):
    yield table
    for child in table.get_children():
        yield from _walk(child)


def test_bench_functions_do_not_shadow_module_imports():
    path = os.path.join(ROOT, "bench.py")
    src = open(path).read()
    imports = _module_imports(ast.parse(src))
    bad = []
    for t in _walk(symtable.symtable(src, path, "exec")):
        if t.get_type() != "function":
            continue
        for sym in t.get_symbols():
            if sym.get_name() in imports and sym.is_local():
                bad.append(f"{t.get_name()}: {sym.get_name()}")
    assert not bad, bad
