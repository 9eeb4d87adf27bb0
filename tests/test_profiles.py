"""The ncu summaries under profiles/ name the commands that made them: every
`bench.py --case NAME` they name is a case bench.py runs, and every
summary gives a command.  Host logic only (no GPU)."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench_cases():
    """Keys of bench.CASES, read from the source (bench.py imports torch)."""
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    for node in tree.body:
        if isinstance(node, ast.Assign) and any(getattr(t, "id", None) == "CASES" for t in node.targets):
            return {k.value for k in node.value.keys}
    raise AssertionError("bench.py defines no CASES")


def _profiles():
    d = os.path.join(ROOT, "profiles")
    return [os.path.join(d, f) for f in sorted(os.listdir(d)) if f.endswith(".md")]


def test_named_cases_exist():
    cases = _bench_cases()
    for p in _profiles():
        for name in re.findall(r"bench\.py --case ([a-z_0-9]+)", open(p).read()):
            assert name in cases, (os.path.basename(p), name)


def test_every_summary_gives_its_command():
    for p in _profiles():
        text = open(p).read()
        assert "ncu " in text and "--clock-control none" in text, os.path.basename(p)


def test_case_functions_are_documented():
    """Each case is a function with a docstring naming its workload."""
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    funcs = {n.name: n for n in tree.body if isinstance(n, ast.FunctionDef)}
    for name in _bench_cases():
        f = funcs.get("case_" + name)
        assert f is not None and ast.get_docstring(f), name
