"""sfci_truncate_topk_noalloc (fixed scratch, no device allocation) against
sfci_truncate_topk on the same inputs, through the C-ABI.

Kept in a file that is collected last so that it also runs after every other
GPU test in the same process; it passes on its own in a fresh process too.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2312_01846_gb300 as sf
    sf.lib()
    return sf


def _input(n, seed):
    rng = np.random.default_rng(seed)
    r = rng.choice(1 << 40, size=n, replace=False).astype(np.uint64)
    # exact ties, exact zeros, both signs, a wide exponent range
    c = rng.choice([0.0, 1.0, -1.0, 0.5, 2.0, -3e-7, 1e-300], size=n) * \
        np.where(rng.random(n) < 0.5, 1.0, rng.random(n))
    return r, c


def test_noalloc_matches_workspace_topk_twice(sf):
    import torch
    cases = [(300_000, 100_000, True, 51), ((1 << 20) + 7, 1 << 20, False, 52)]
    kmax = max(k for _, k, _, _ in cases)
    out_r = torch.empty(kmax, dtype=torch.int64, device="cuda")
    out_c = torch.empty(kmax, dtype=torch.float64, device="cuda")
    # first call: sets up the scratch address for this device
    r0, c0 = _input(1000, 50)
    sf.sfci_truncate_topk_noalloc(r0, c0, 10, True, out_r, out_c)
    for n, k, norm, seed in cases:
        r, c = _input(n, seed)
        rd = torch.from_numpy(r.view(np.int64)).cuda()
        cd = torch.from_numpy(c).cuda()
        wr, wv = sf.sfci_truncate_topk(rd, cd, k, normalize=norm)
        wr, wv = wr.clone(), wv.clone()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        gr, gv = sf.sfci_truncate_topk_noalloc(rd, cd, k, norm, out_r, out_c)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert gr.numel() == wr.numel()
        assert torch.equal(gr, wr)
        if norm:
            assert np.allclose(gv.cpu().numpy(), wv.cpu().numpy(), rtol=1e-15, atol=0)
        else:
            assert np.array_equal(gv.cpu().numpy().view(np.uint64), wv.cpu().numpy().view(np.uint64))


def test_noalloc_rejects_k_above_scratch(sf):
    import torch
    r, c = _input(100, 53)
    rd = torch.from_numpy(r.view(np.int64)).cuda()
    cd = torch.from_numpy(c).cuda()
    n = C.c_int64()
    st = sf.lib().sfci_truncate_topk_noalloc(sf._ptr(rd), sf._ptr(cd), 100, (1 << 20) + 1, 1,
                                             sf._ptr(rd), sf._ptr(cd), C.byref(n), sf._stream())
    assert st == sf.SFCI_E_CAPACITY
    assert "1048576" in sf.lib().sfci_last_error().decode()
