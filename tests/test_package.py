"""The package without a GPU: the product path never touches the oracle and fails loudly
without its CUDA library; the reference arm's JSON line carries the contract's keys."""
import ast
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2401_16378_gb300")


def test_product_code_never_imports_the_oracle():
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            if not f.endswith(".py"):
                continue
            tree = ast.parse(open(os.path.join(dirpath, f)).read())
            for node in ast.walk(tree):
                names = []
                if isinstance(node, ast.Import):
                    names = [a.name for a in node.names]
                elif isinstance(node, ast.ImportFrom):
                    names = [node.module or ""]
                assert not any(n == "oracle" or n.startswith("oracle.") for n in names), (f, names)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2401_16378_gb300 import _lib

    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libpauli.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        _lib.load()


def test_reference_arm_line_has_the_contract_keys():
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--qubits", "8"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["vs_baseline"] is None and d["higher_is_better"] is True
    assert "workload" in d["config"]
    assert set(d["cpu_baseline"]) >= {"value", "unit", "cores", "kind", "sample"}
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_every_binding_is_exported_by_the_package():
    """Each pauli_* binding in api.py, and its short alias, is reachable from the package."""
    import inspect

    import paper_2401_16378_gb300 as pg
    from paper_2401_16378_gb300 import api

    names = [n for n, f in inspect.getmembers(api, inspect.isfunction)
             if n.startswith("pauli_") and f.__module__ == api.__name__]
    assert "pauli_decompose_xhi" in names
    for n in names:
        assert hasattr(pg, n), n
        short = n[len("pauli_"):]
        if hasattr(api, short):
            assert hasattr(pg, short), short
