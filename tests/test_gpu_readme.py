"""The README's quick-start block runs as written and gives what its comments say."""
import os
import re

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_quick_start_runs(tmp_path, monkeypatch):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_03413_gb300 import build
    build.build()
    text = open(os.path.join(ROOT, "README.md")).read()
    block = re.search(r"```python\n(.*?)```", text, re.S).group(1)
    ns = {}
    monkeypatch.chdir(tmp_path)  # files the example writes (its tuning cache) land here
    exec(compile(block, "README.md", "exec"), ns)
    torch.cuda.synchronize()
    cw = ns["cw"]
    assert ns["rc"] == cw.CW_OK and ns["stats"].rel_residual <= 1e-10
    assert torch.isfinite(ns["y"]).all()
    # the batched results equal the per-operator apply of each right-hand side
    for o, x, y in zip(ns["ops"], ns["xs"], ns["ys"]):
        for r in range(x.shape[0]):
            assert torch.equal(y[r], o.apply(x[r]))
    # the multigrid solve converges in a handful of V-cycles; the two-block solve converges
    assert ns["mg_rc"] == cw.CW_OK and ns["mg_stats"].rel_residual <= 1e-10 and ns["mg_stats"].iterations <= 20
    assert ns["mb_rc"] == cw.CW_OK and ns["mb_stats"].rel_residual <= 1e-10
    assert ns["mb"].shared_dofs()[0] > 0  # the glued face's interior DoFs
    assert (tmp_path / "tune.json").exists()
