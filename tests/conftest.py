import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def pytest_terminal_summary(terminalreporter):
    """Recall@k and the largest relative distance error of every checked
    full-size result, one line each (recorded by the GPU tests)."""
    mod = sys.modules.get("tests.parity")
    summary = getattr(mod, "SUMMARY", None)
    if not summary:
        return
    terminalreporter.section("parity against the oracle")
    for name, (rows, rec, err) in sorted(summary.items()):
        terminalreporter.write_line(f"{name}: {rows} rows, recall@k {rec:.6f}, "
                                    f"max rel dist err {err:.2e}")
