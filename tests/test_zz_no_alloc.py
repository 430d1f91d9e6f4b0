"""The allocation-free descriptor range (nep_descriptor_range_noalloc) agrees with the
regular entry point.

That entry point exists for callers that cannot allocate device memory during a call
(inside CUDA-graph stream capture, under a host-owned memory manager, or in loops that
must stay out of the allocator); it keeps its scratch in a fixed array inside the
library.  This file is named to run last: it checks two calls in a row through the C
ABI, and it must also pass on its own in a fresh process, where the first call does the
one-time lookup of the scratch array's device address.
"""
import ctypes

import numpy as np
import pytest

from paper_2606_19557_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def test_noalloc_descriptor_range_matches_regular_entry_point():
    from paper_2606_19557_gb300 import NEP
    spec = synth.SPECS["fcc_bcc_t1"]
    batch = synth.batch_fcc_bcc(seed=21, n_struct=12)
    nep = NEP(spec)
    nep.set_structures_batch(batch)
    theta = torch.tensor(synth.random_theta(nep.P, 3), dtype=torch.float32)
    nep.set_params(theta, torch.ones(nep.n_des))
    lo_ref, hi_ref = [x.cpu().numpy() for x in nep.descriptor_range()]

    fn = nep.lib.nep_descriptor_range_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    for _ in range(2):  # two calls in a row share (and overwrite) the scratch array
        lo = torch.full((nep.n_des,), float("nan"), dtype=torch.float32, device="cuda")
        hi = torch.full((nep.n_des,), float("nan"), dtype=torch.float32, device="cuda")
        nep._enter()
        rc = fn(nep.h, ctypes.c_void_p(lo.data_ptr()), ctypes.c_void_p(hi.data_ptr()))
        nep._leave()
        assert rc == 0, nep.lib.nep_last_error(nep.h).decode()
        torch.cuda.synchronize()
        np.testing.assert_allclose(lo.cpu().numpy(), lo_ref, rtol=TOL, atol=0)
        np.testing.assert_allclose(hi.cpu().numpy(), hi_ref, rtol=TOL, atol=0)


def test_noalloc_and_regular_range_match_oracle_descriptors():
    """Both entry points against the per-component minimum and maximum of the oracle's raw
    descriptors (before the scale of Eq. "norm") on the same batch."""
    import oracle
    from paper_2606_19557_gb300 import NEP
    spec = synth.SPECS["alloy_t4"]
    batch = synth.batch_alloy(seed=22, n_struct=10)
    nep = NEP(spec)
    nep.set_structures_batch(batch)
    theta = synth.random_theta(nep.P, 4)
    nep.set_params(torch.tensor(theta, dtype=torch.float32), torch.ones(nep.n_des))
    q = oracle.descriptors(spec, theta, batch)
    scale = np.abs(q).max()
    lo, hi = [x.cpu().numpy() for x in nep.descriptor_range()]
    np.testing.assert_allclose(lo, q.min(axis=0), rtol=TOL, atol=1e-6 * scale)
    np.testing.assert_allclose(hi, q.max(axis=0), rtol=TOL, atol=1e-6 * scale)
    fn = nep.lib.nep_descriptor_range_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lo2 = torch.empty(nep.n_des, dtype=torch.float32, device="cuda")
    hi2 = torch.empty(nep.n_des, dtype=torch.float32, device="cuda")
    nep._enter()
    assert fn(nep.h, ctypes.c_void_p(lo2.data_ptr()), ctypes.c_void_p(hi2.data_ptr())) == 0
    nep._leave()
    torch.cuda.synchronize()
    np.testing.assert_allclose(lo2.cpu().numpy(), q.min(axis=0), rtol=TOL, atol=1e-6 * scale)
    np.testing.assert_allclose(hi2.cpu().numpy(), q.max(axis=0), rtol=TOL, atol=1e-6 * scale)
    nep.close()


def test_noalloc_rejects_batches_above_its_scratch_size():
    """A batch whose atoms x padded descriptor length exceed the fixed scratch array
    (8,388,608 floats) is rejected with NEP_EINVAL, the limit named in the message, and the
    outputs left untouched; the regular entry point, which allocates, still serves it."""
    from paper_2606_19557_gb300 import NEP, NEP_EINVAL
    spec = synth.SPECS["fcc_bcc_t1"]
    batch = synth.batch_fcc_bcc(seed=23, n_struct=1700)
    assert batch.n_atoms * (5 + 6 * 5) > 8_388_608  # padded descriptor length of this model: 35
    nep = NEP(spec)
    nep.set_structures_batch(batch)
    nep.set_params(torch.tensor(synth.random_theta(nep.P, 5), dtype=torch.float32), torch.ones(nep.n_des))
    fn = nep.lib.nep_descriptor_range_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lo = torch.full((nep.n_des,), float("nan"), dtype=torch.float32, device="cuda")
    hi = torch.full((nep.n_des,), float("nan"), dtype=torch.float32, device="cuda")
    nep._enter()
    rc = fn(nep.h, ctypes.c_void_p(lo.data_ptr()), ctypes.c_void_p(hi.data_ptr()))
    nep._leave()
    assert rc == NEP_EINVAL
    assert "8388608" in nep.lib.nep_last_error(nep.h).decode().replace(",", "")
    torch.cuda.synchronize()
    assert torch.isnan(lo).all() and torch.isnan(hi).all()
    lo_ref, hi_ref = nep.descriptor_range()
    assert torch.isfinite(lo_ref).all() and torch.isfinite(hi_ref).all()
    nep.close()
