"""kete_propagate_noalloc: propagation for callers that cannot allocate device
memory while they run (their GPU memory is handed to their own pool at
start-up, or a real-time thread must not block in the driver's allocator).

The entry point is called through the C ABI and compared with kete_propagate,
the allocating entry point it mirrors, on two calls in a row with different
targets, so that a stop epoch left in the shared device array by the first
call would show in the second.
This file is collected last so a failure here does not hide the others."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

POS_TOL = 1e-9    # AU, the position tolerance of the propagation parity tests
VEL_TOL = 1e-11   # AU/day


def test_noalloc_matches_propagate_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_04666_gb300 import build as B, kete, workloads as W
    B.build()
    w = W.propagation_only("noalloc", 4000, 40.0, 0, n_neo=400)
    n = w.n_bodies
    K = kete.Kete(0)
    K.load_ephem(w.ephem.to_bytes())
    L = kete.lib()
    fm = kete.force_model()
    for call, t1 in enumerate((W.T0 + 7.5, W.T0 + 31.25)):
        ref_st = torch.from_numpy(w.states.copy()).cuda()
        ref_ep = torch.from_numpy(w.epochs.copy()).cuda()
        ref_status = torch.zeros(n, dtype=torch.int32, device="cuda")
        rc = L.kete_propagate(K._h, ref_st.data_ptr(), ref_ep.data_ptr(), n, t1, C.byref(fm),
                              ref_status.data_ptr())
        assert rc == kete.OK
        st = torch.from_numpy(w.states.copy()).cuda()
        ep = torch.from_numpy(w.epochs.copy()).cuda()
        status = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        rc = L.kete_propagate_noalloc(K._h, st.data_ptr(), ep.data_ptr(), n, t1, C.byref(fm),
                                      status.data_ptr())
        assert rc == kete.OK, L.kete_last_error(K._h)
        torch.cuda.synchronize()
        assert (status.cpu() == 0).all() and (ref_status.cpu() == 0).all()
        assert (ep.cpu().numpy() == t1).all()
        a, b = st.cpu().numpy(), ref_st.cpu().numpy()
        assert np.abs(a[:3] - b[:3]).max() <= POS_TOL, call
        assert np.abs(a[3:] - b[3:]).max() <= VEL_TOL, call
        assert not np.array_equal(a, w.states)
    # sizes beyond the fixed array are refused with a clear message
    big = kete.NOALLOC_MAX_BODIES + 1
    rc = L.kete_propagate_noalloc(K._h, st.data_ptr(), ep.data_ptr(), big, W.T0 + 1.0,
                                  C.byref(fm), status.data_ptr())
    assert rc == kete.ERR_BAD_ARG
    assert b"KETE_NOALLOC_MAX_BODIES" in L.kete_last_error(K._h)
    K.close()
