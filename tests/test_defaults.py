"""The oracle keeps its own table of parameter defaults (it imports nothing
from the CUDA package); this checks that the two tables name the same
parameters with the same values, so that a change on either side fails here
instead of silently moving one implementation away from the other."""


def test_oracle_and_library_defaults_agree():
    from oracle.oracle import DEFAULTS
    from paper_2004_04080_gb300.workloads import default_params

    lib = default_params()
    assert sorted(DEFAULTS) == sorted(lib)
    for k, v in DEFAULTS.items():
        assert tuple(v) == tuple(lib[k]) if isinstance(v, tuple) else v == lib[k], k


def test_oracle_imports_nothing_from_the_package():
    import ast
    import os

    root = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")
    for name in os.listdir(root):
        if not name.endswith(".py"):
            continue
        tree = ast.parse(open(os.path.join(root, name)).read())
        for node in ast.walk(tree):
            mods = []
            if isinstance(node, ast.Import):
                mods = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                mods = [node.module or ""]
            for m in mods:
                assert not m.startswith("paper_2004_04080_gb300"), (name, m)
