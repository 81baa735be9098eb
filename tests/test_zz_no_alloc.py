"""kfmm_direct_noalloc: the all-pairs direct sum for callers that cannot allocate device
memory (a process whose memory already sits in a caching allocator, or code that must not
call cudaMalloc / cudaFree while running because those calls synchronise the device).

It must agree with kfmm_direct, the allocating entry point, within the tolerances the other
direct-sum tests use (FP64 1e-12, FP32 3e-5 relative L2), on two calls in a row: the second
call runs on scratch memory that still holds the first call's partial sums.

This file is named to be collected last, so a run that stops at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def K():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_04082_gb300 as K
    return K


def rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def case(rng, ns, nt, dtype):
    src = torch.tensor(rng.uniform(-1, 1, (ns, 3)), dtype=dtype, device="cuda")
    trg = torch.cat([torch.tensor(rng.uniform(-1, 1, (nt - 3, 3)), dtype=dtype, device="cuda"), src[:3]])
    nrm = rng.normal(size=(ns, 3))
    nrm = torch.tensor(nrm / np.linalg.norm(nrm, axis=1, keepdims=True), dtype=dtype, device="cuda")
    sl = torch.tensor(rng.normal(size=(ns, 3)), dtype=dtype, device="cuda")
    dl = torch.tensor(rng.normal(size=(ns, 3)), dtype=dtype, device="cuda")
    return trg.contiguous(), src, nrm, sl, dl


def test_noalloc_matches_direct_on_two_calls(K):
    rng = np.random.default_rng(21)
    with K.Kfmm() as f:
        f.set_material(K.material_K(2.3, 0.21), 2.3)
        calls = [
            # (precision, torch dtype, kind, n_src, n_trg, tolerance, layers)
            (K.KFMM_FP32, torch.float32, K.KFMM_DISP, 20011, 37, 3e-5, "sl+dl"),
            (K.KFMM_FP64, torch.float64, K.KFMM_STRESS, 3001, 1299, 1e-12, "sl+dl"),
            # every other instantiation: single and double layer alone, FP32 stress
            (K.KFMM_FP32, torch.float32, K.KFMM_DISP, 5003, 211, 3e-5, "sl"),
            (K.KFMM_FP32, torch.float32, K.KFMM_DISP, 5003, 211, 3e-5, "dl"),
            (K.KFMM_FP32, torch.float32, K.KFMM_STRESS, 4001, 301, 3e-5, "sl+dl"),
            (K.KFMM_FP64, torch.float64, K.KFMM_DISP, 2003, 97, 1e-12, "dl"),
        ]
        for prec, dt, kind, ns, nt, tol, layers in calls:
            trg, src, nrm, sl, dl = case(rng, ns, nt, dt)
            if layers == "sl":
                dl = None
            elif layers == "dl":
                sl = None
            no = 3 if kind == K.KFMM_DISP else 6
            ref = torch.zeros(nt, no, dtype=dt, device="cuda")
            f.direct(trg, src, nrm, sl, dl, ref, kind, prec)
            got = torch.full((nt, no), float("nan"), dtype=dt, device="cuda")
            K.kfmm_direct_noalloc(f.handle, trg, src, nrm, sl, dl, got, kind, prec)
            torch.cuda.synchronize()
            assert torch.isfinite(got).all()
            assert rel(got, ref) < tol, (prec, kind, layers)


def test_noalloc_rejects_oversize_and_host_arrays(K):
    with K.Kfmm() as f:
        n = (16 << 20) // 12 + 1  # one FP32 displacement target more than the scratch holds
        trg = torch.zeros(n, 3, device="cuda")
        src = torch.ones(4, 3, device="cuda")
        den = torch.ones(4, 3, device="cuda")
        out = torch.zeros(n, 3, device="cuda")
        with pytest.raises(K.KfmmError) as e:
            K.kfmm_direct_noalloc(f.handle, trg, src, None, den, None, out)
        assert e.value.status == K.KFMM_ERR_INVALID_ARG
        with pytest.raises(K.KfmmError) as e:
            K.kfmm_direct_noalloc(f.handle, trg[:8].cpu(), src, None, den, None, out[:8])
        assert e.value.status == K.KFMM_ERR_INVALID_ARG
