"""The per-step JSON log (SFCI_STEP_LOG): one parseable line per solver step
carrying the same scalars as the step's info."""
import json
import os

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2312_01846_gb300 as sf
    sf.lib()
    return sf


def test_step_log_lines(sf, tmp_path):
    path = tmp_path / "steps.jsonl"
    os.environ["SFCI_STEP_LOG"] = str(path)
    try:
        gsys = sf.System.from_dict(gen.config_system(0))
        lz = sf.Lanczos(gsys, np.array([0], dtype=np.uint64), np.array([1.0]), 300, 5)
        infos = [lz.step() for _ in range(7)]
        lz.close()
        gsys.close()
    finally:
        del os.environ["SFCI_STEP_LOG"]
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert len(lines) == 7
    for got, info in zip(lines, infos):
        for k in ("iter", "cycle", "index", "cycle_end", "n_in", "n_sigma", "n_elements", "n_emitted"):
            assert got[k] == info[k], k
        assert got["a"] == info["a"] and got["lambda_min"] == info["lambda_min"]
        assert got["sigma_gbs_32B_per_element"] > 0.0
    assert sum(x["cycle_end"] for x in lines) == 1


def test_set_input_keeps_the_cycle(sf):
    """A run whose every input vector makes a round trip through host memory
    and sfci_lanczos_set_input equals, bit for bit, the run that keeps its
    vectors on the device (the cycle, T and S carry on)."""
    import torch
    d = gen.config_system(2)
    gsys = sf.System.from_dict(d)
    ref = sf.Lanczos(gsys, np.array([0], dtype=np.uint64), np.array([1.0]), 3000, 4)
    infos_ref = [ref.step() for _ in range(9)]
    r_ref, c_ref = ref.vector()
    ref.close()
    lz = sf.Lanczos(gsys, np.array([0], dtype=np.uint64), np.array([1.0]), 3000, 4)
    infos = []
    for _ in range(9):
        r, c = lz.vector()
        hr, hc = r.cpu().pin_memory(), c.cpu().pin_memory()
        lz.set_input(hr.cuda(), hc.cuda())
        infos.append(lz.step())
    r2, c2 = lz.vector()
    lz.close()
    gsys.close()
    for key in ("a", "b", "lambda_min", "n_kept", "cycle_end"):
        assert [i[key] for i in infos] == [i[key] for i in infos_ref], key
    assert torch.equal(r2, r_ref) and torch.equal(c2, c_ref)
    with pytest.raises(sf.SfciError):
        g2 = sf.System.from_dict(d)
        z = sf.Lanczos(g2, np.array([0], dtype=np.uint64), np.array([1.0]), 10, 4)
        try:
            z.set_input(np.arange(11, dtype=np.uint64), np.ones(11))
        finally:
            z.close()
            g2.close()
