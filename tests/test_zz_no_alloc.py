"""The allocation-free gradient entry point, against the oracle and the allocating one.

hydro_mlp_loss_grad_device is for callers that must not allocate device
memory while they call in: a host framework that owns all of the GPU's memory
through its own pool, or a code whose memory budget is fixed when it starts.
Its scratch is a static device array.  On two calls in a row that reuse that
array it must give the gradient and loss of the FP64 CPU oracle's backprop
(oracle.mlp_loss_grad) within the tolerance the gradient tests use (1e-4 of
the gradient norm, 1e-5 of the loss), agree with hydro_mlp_loss_grad to the
same bar, and reject sizes beyond the array.  This file sorts last so that a
failure here comes after every other test has run.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


def _device_grad(H, torch, w, X, T):
    n = len(T)
    dw = torch.from_numpy(w).cuda()
    dx = torch.from_numpy(X.astype(np.float32)).cuda()
    dt = torch.from_numpy(T.astype(np.float32)).cuda()
    dg = torch.full((H.HYDRO_MLP_NPARAM,), np.nan, dtype=torch.float64, device="cuda")
    dl = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    H.hydro_mlp_loss_grad_device(dw.data_ptr(), dx.data_ptr(), dt.data_ptr(), n, dg.data_ptr(), dl.data_ptr(),
                                 stream.cuda_stream)
    torch.cuda.synchronize()
    return float(dl.item()), dg.cpu().numpy()


def test_device_gradient_matches_oracle_and_allocating_entry_point(hydro_lib):
    import torch
    H = hydro_lib
    rng = np.random.default_rng(77)
    w = (0.3 * rng.standard_normal(H.HYDRO_MLP_NPARAM)).astype(np.float32)
    # two calls in a row on the same scratch: a larger one, then a smaller one
    # (the second reads none of the first call's partials)
    for n in (H.HYDRO_NOALLOC_MAX_SAMPLES, 333):
        X = rng.normal(size=(n, 6)).astype(np.float32).astype(np.float64)
        T = rng.normal(size=n).astype(np.float32).astype(np.float64)
        loss_o, g_o = O.mlp_loss_grad(w, X, T)
        loss, g = _device_grad(H, torch, w, X, T)
        assert np.all(np.isfinite(g))
        assert abs(loss - loss_o) <= 1e-5 * loss_o, (n, loss, loss_o)
        err = np.linalg.norm(g - g_o) / np.linalg.norm(g_o)
        print("n=%d: |g - g_oracle| / |g_oracle| = %.3e" % (n, err))
        assert err <= 1e-4, n
        loss_ref, g_ref = H.hydro_mlp_loss_grad(w, X, T)
        assert abs(loss - loss_ref) <= 1e-5 * loss_ref
        assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref), n


def test_device_gradient_rejects_sizes_beyond_its_scratch(hydro_lib):
    import torch
    H = hydro_lib
    n = H.HYDRO_NOALLOC_MAX_SAMPLES + 1
    buf = torch.zeros(max(6 * n, H.HYDRO_MLP_NPARAM), dtype=torch.float64, device="cuda")
    with pytest.raises(H.HydroError) as e:
        H.hydro_mlp_loss_grad_device(buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), n, buf.data_ptr(),
                                     buf.data_ptr(), None)
    assert e.value.status == H.HYDRO_ERR_ARG
    assert "16384" in str(e.value)
