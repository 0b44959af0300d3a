"""The library for host-only tests (no GPU): built in-tree first if needed,
then imported.  Only calls that make no CUDA call are used through it."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def mica():
    spec = importlib.util.spec_from_file_location("mica_build", os.path.join(ROOT, "paper_1402_4876_gb300", "_build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    import paper_1402_4876_gb300 as m
    return m
