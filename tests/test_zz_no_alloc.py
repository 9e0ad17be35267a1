"""tn_absorb_dot_noalloc against tn_absorb_dot, through the C-ABI.

The no-allocation entry point serves callers that must not call the CUDA
allocator where they call the library (latency-critical loops, processes whose
device memory another allocator already holds); its scratch is a fixed array
inside the library.  Two calls in a row must both agree with the allocating
entry point: the second call finds the first call's partials still in the
array and must clear what has to start at zero.  This file is collected last
so a run that stops at the first failure has already run every other test.
"""
import pytest

from paper_1908_08553_gb300 import tn

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("K,N,P,S", [(16, 16, 7, 1000), (81, 81, 3, 300), (4, 16, 1, 4096), (16, 4, 33, 1)])
def test_noalloc_matches_allocating_entry_point(dtype, K, N, P, S):
    import torch
    tdt = torch.float64 if dtype == 0 else torch.float32
    g = torch.Generator().manual_seed(11 * K + N + P + S)
    x = (torch.rand(P, K, S, generator=g, dtype=torch.float64) * 2 - 1).to(tdt).cuda()
    E = (torch.rand(K, N, generator=g, dtype=torch.float64) * 2 - 1).to(tdt).cuda()
    adj = (torch.rand(P, N, S, generator=g, dtype=torch.float64) * 2 - 1).to(tdt).cuda()
    scale = float(torch.einsum("pks,kn,pns->", x.double().abs(), E.double().abs(), adj.double().abs()))
    st = torch.cuda.current_stream()
    ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    got = torch.zeros(2, dtype=torch.float64, device="cuda")
    tn.tn_absorb_dot(dtype, x, E, adj, P, K, N, S, ref, st)
    tn.tn_absorb_dot_noalloc(dtype, x, E, adj, P, K, N, S, got[0:1], st)
    tn.tn_absorb_dot_noalloc(dtype, x, E, adj, P, K, N, S, got[1:2], st)
    torch.cuda.synchronize()
    tol = 1e-13 if dtype == 0 else 1e-6
    r = float(ref.item())
    for v in got.cpu().tolist():
        assert abs(v - r) <= tol * scale, (v, r)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(tn.TNError) as e:
        # 2^24 + 1 outer positions: one tile more than the fixed array holds
        tn.tn_absorb_dot_noalloc(1, x, x, x, 1, 16, 16, 2 ** 24 + 1, out, torch.cuda.current_stream())
    assert e.value.status == tn.TN_ERR_INVALID
