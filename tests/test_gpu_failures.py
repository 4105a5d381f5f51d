"""Failure paths of the C ABI, made to happen without faulting the GPU.

* a NaN in the site tensor, written on the host before the copy: the spectra come out
  non-finite and the call returns CTM_ERR_NONFINITE;
* a Jacobi sweep limit of 1 set on the handle: the SVD stops unconverged and the call returns
  CTM_ERR_SVD_NOCONV;
* a spin limit of 1 set on the handle: the first block that has to wait at a grid barrier of
  the cooperative QR / Jacobi kernels gives up at once, tells the other blocks to stop, and the
  call returns CTM_ERR_TIMEOUT.

Every wait in those kernels is bounded, so nothing here hangs or faults; after each error the
same handle is re-initialised and must evaluate normally again.
"""
import math

import pytest
import torch

import workloads as W
from gpu_helpers import env_flat, make_ctm, site_stack

pytestmark = pytest.mark.gpu

NONFINITE, SVD_NOCONV, TIMEOUT = 4, 5, 7


def _recovers(ctm, w):
    ctm.set_limits(0, 0)
    ctm.init(site_stack(w.tensors), env_flat(W.initial_environment(w)))
    ctm.step(2)
    e = float(ctm.energy()[0])
    assert math.isfinite(e)
    return e


def test_nan_site_tensor_reports_nonfinite_and_handle_recovers():
    from paper_2512_14414_gb300 import CTMError
    w = W.config("heis_d2_chi8")
    ctm = make_ctm(w)
    A = site_stack(w.tensors).cpu()
    A[0, 1, 0, 1, 0, 1] = float("nan")
    ctm.init(A.cuda(), env_flat(W.initial_environment(w)))
    with pytest.raises(CTMError) as ei:
        ctm.step(2)
    assert ei.value.status == NONFINITE
    e = _recovers(ctm, w)
    ref = make_ctm(w)
    ref.init(site_stack(w.tensors), env_flat(W.initial_environment(w)))
    ref.step(2)
    assert e == float(ref.energy()[0])


def test_sweep_limit_reports_svd_noconv():
    from paper_2512_14414_gb300 import CTMError
    w = W.config("heis_d4_chi32")
    ctm = make_ctm(w)
    ctm.set_limits(max_sweeps=1)
    ctm.init(site_stack(w.tensors), env_flat(W.initial_environment(w)))
    with pytest.raises(CTMError) as ei:
        ctm.step(1)
    assert ei.value.status == SVD_NOCONV
    _recovers(ctm, w)


def test_short_wait_limit_reports_timeout():
    from paper_2512_14414_gb300 import CTMError
    w = W.config("heis_d4_chi32")
    ctm = make_ctm(w)
    ctm.set_limits(spin_limit=1)
    ctm.init(site_stack(w.tensors), env_flat(W.initial_environment(w)))
    with pytest.raises(CTMError) as ei:
        ctm.step(1)
    assert ei.value.status == TIMEOUT
    torch.cuda.synchronize()  # the context is still usable
    _recovers(ctm, w)
