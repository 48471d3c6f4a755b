"""ksc_prox_g_noalloc -- the prox entry point for callers that cannot allocate
device memory (runtimes that own all device memory through their own pools,
loops that cannot take an allocation's implicit synchronisation) -- must return
what the allocating ksc_prox_g returns, call after call, although every call
reuses the same fixed device scratch array.  The file is named to be collected
last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    import __graft_entry__ as g
    g.build()
    from paper_2502_09502_gb300 import ksc
    return ksc


@pytest.mark.parametrize("p,k,want_top", [(50000, 20, True), (3001, 7, True), (50000, 33, False)])
def test_noalloc_prox_matches_allocating_prox_on_consecutive_calls(K, p, k, want_top):
    # p = 50000 does not fit in shared memory: the kernel keeps its copy of w in
    # the fixed device scratch array
    import torch
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(1000 + p + k)
    rho, M = 2.5, 1.3
    for call in range(2):        # the second call must not see the first call's scratch
        w = rng.standard_normal(p) * (0.5 + call)
        ref_beta, ref_top = K.ksc_prox_g(w, k, M, rho)
        wd = torch.from_numpy(w).cuda()
        bd = torch.full_like(wd, float("nan"))
        td = torch.full((k,), -1, dtype=torch.int32, device="cuda")
        st = K.ksc_prox_g_noalloc(wd.data_ptr(), p, k, M, rho, bd.data_ptr(),
                                  td.data_ptr() if want_top else None, stream)
        assert st == K.KSC_OK, K.ksc_last_error()
        torch.cuda.synchronize()
        beta = bd.cpu().numpy()
        assert np.max(np.abs(beta - ref_beta)) <= 1e-11 * max(1.0, np.abs(w).max())
        if want_top:
            assert np.array_equal(td.cpu().numpy(), ref_top)


def test_noalloc_prox_rejects_sizes_beyond_its_scratch(K):
    # the size check comes before any device access
    st = K.ksc_prox_g_noalloc(16, (1 << 19) + 1, 5, 1.0, 1.0, 16, None, None)
    assert st == K.KSC_ERR_INVALID_ARG
    assert "allocation-free maximum" in K.ksc_last_error()
