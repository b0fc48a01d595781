"""The allocation-free field entry point (md_coulomb_field_device_noalloc).

Some callers cannot allocate device memory: code running inside another
framework's memory pool, a CUDA-graph builder that must not see cudaMalloc, a
plugin whose host forbids allocation.  For them the library offers a field
evaluation whose scratch memory is a fixed array compiled into the library.
This test calls it through the C ABI twice in a row and checks each result
against the allocating entry point md_coulomb_field_device and against the
FP64 oracle's direct sum, within the same tolerance as the other field tests;
a third case fills the scratch array to its 32768-target limit.  The file sits
on its own, collected last, and works both alone in a fresh process and after
the other tests.
"""
import os

import numpy as np
import pytest

import oracle
from tests.helpers import force_error, summary

pytestmark = pytest.mark.gpu

FORCE_P99 = 2e-5
MAX_TARGETS = 32768
NTHREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def md():
    from paper_1307_3711_gb300 import build
    build.build()
    from paper_1307_3711_gb300 import md as m
    return m


def _field(md, fn, src, ns, tgt, nt, eps2, self_offset, stream):
    import torch
    e = torch.full((nt, 3), float("nan"), dtype=torch.float64, device="cuda")
    phi = torch.full((nt,), float("nan"), dtype=torch.float64, device="cuda")
    fn(src.data_ptr(), ns, tgt.data_ptr(), nt, eps2, self_offset, e.data_ptr(), phi.data_ptr(),
       stream)
    torch.cuda.synchronize()
    return e.cpu().numpy(), phi.cpu().numpy()


def test_noalloc_field_matches_allocating_entry_point_twice(md):
    import torch
    kc = oracle.coulomb_constant(0.8)
    stream = torch.cuda.current_stream().cuda_stream
    eps = 1e-3
    rng = np.random.default_rng(21)
    # first call: separate targets, sources split into several segments
    ns, nt = 21001, 3001
    xs = rng.normal(size=(ns, 3)) * 0.02
    qs = rng.choice([-1.0, 1.0, 3.0], size=ns)
    xt = rng.normal(size=(nt, 3)) * 0.02
    src = torch.tensor(np.c_[xs, kc * qs], dtype=torch.float32, device="cuda")
    tgt = torch.tensor(np.c_[xt, np.zeros(nt)], dtype=torch.float32, device="cuda")
    ref = _field(md, md.coulomb_field_device, src, ns, tgt, nt, eps * eps, -1, stream)
    got = _field(md, md.coulomb_field_device_noalloc, src, ns, tgt, nt, eps * eps, -1, stream)
    assert md.field_device_status(stream) == md.MD_OK
    assert summary(force_error(got[0], ref[0]))["p99"] <= FORCE_P99
    np.testing.assert_allclose(got[1], ref[1], rtol=1e-5, atol=1e-5 * np.abs(ref[1]).max())
    e64, phi64 = oracle.coulomb_field(xt, xs, qs, eps, kc, potential=True, nthreads=NTHREADS)
    assert summary(force_error(got[0], e64))["p99"] <= FORCE_P99
    np.testing.assert_allclose(got[1], phi64, rtol=1e-5, atol=1e-5 * np.abs(phi64).max())
    # second call in a row: targets are the sources (self term removed)
    ns2 = 9000
    src2 = src[:ns2].clone()
    ref = _field(md, md.coulomb_field_device, src2, ns2, src2, ns2, eps * eps, 0, stream)
    got = _field(md, md.coulomb_field_device_noalloc, src2, ns2, src2, ns2, eps * eps, 0, stream)
    assert md.field_device_status(stream) == md.MD_OK
    assert summary(force_error(got[0], ref[0]))["p99"] <= FORCE_P99
    np.testing.assert_allclose(got[1], ref[1], rtol=1e-5, atol=1e-5 * np.abs(ref[1]).max())
    e64, phi64 = oracle.self_field(xs[:ns2], qs[:ns2], eps, kc, potential=True, nthreads=NTHREADS)
    assert summary(force_error(got[0], e64))["p99"] <= FORCE_P99
    np.testing.assert_allclose(got[1], phi64, rtol=1e-4, atol=2e-5 * np.abs(phi64).max())


def test_noalloc_field_at_its_target_limit(md):
    """nt = 32768 uses every completion counter and the top rows of each
    segment's partials; 8192 sources make 4 segments."""
    import torch
    kc = oracle.coulomb_constant(0.8)
    stream = torch.cuda.current_stream().cuda_stream
    eps = 1e-3
    rng = np.random.default_rng(22)
    ns, nt = 8192, MAX_TARGETS
    xs = rng.uniform(-0.02, 0.02, size=(ns, 3))
    qs = rng.choice([-1.0, 2.0], size=ns)
    xt = rng.uniform(-0.02, 0.02, size=(nt, 3))
    src = torch.tensor(np.c_[xs, kc * qs], dtype=torch.float32, device="cuda")
    tgt = torch.tensor(np.c_[xt, np.zeros(nt)], dtype=torch.float32, device="cuda")
    ref = _field(md, md.coulomb_field_device, src, ns, tgt, nt, eps * eps, -1, stream)
    got = _field(md, md.coulomb_field_device_noalloc, src, ns, tgt, nt, eps * eps, -1, stream)
    assert md.field_device_status(stream) == md.MD_OK
    assert np.isfinite(got[0]).all() and np.isfinite(got[1]).all()
    assert summary(force_error(got[0], ref[0]))["p99"] <= FORCE_P99
    e64, phi64 = oracle.coulomb_field(xt, xs, qs, eps, kc, potential=True, nthreads=NTHREADS)
    assert summary(force_error(got[0], e64))["p99"] <= FORCE_P99
    np.testing.assert_allclose(got[1], phi64, rtol=1e-5, atol=1e-5 * np.abs(phi64).max())


def test_noalloc_rejects_too_many_targets(md):
    import torch
    src = torch.zeros((16, 4), dtype=torch.float32, device="cuda")
    tgt = torch.zeros((MAX_TARGETS + 1, 4), dtype=torch.float32, device="cuda")
    e = torch.zeros((MAX_TARGETS + 1, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(md.MDError) as ei:
        md.coulomb_field_device_noalloc(src.data_ptr(), 16, tgt.data_ptr(), MAX_TARGETS + 1,
                                        1e-6, -1, e.data_ptr(), 0, 0)
    assert ei.value.status == md.MD_ERR_ARG
    assert "32768" in str(ei.value)
