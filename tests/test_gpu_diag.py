"""Diagnostics entry points on the GPU: the double-float logarithm of the
mixed form's micro law against CUDA's float64 log, and the execution-unit
throughput probes that give the roofline denominators."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
rv = pytest.importorskip('paper_2306_02687_gb300')


def _df_round(x):
    """x rounded to the double-float pair (hi, lo) the kernel forms from it."""
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    return hi.astype(np.float64) + lo.astype(np.float64)


@pytest.mark.parametrize('lo,hi,tol', [(0.5, 2.0, 3e-14), (1e-6, 1e6, 3e-14)])
def test_df_log_against_float64_log(lo, hi, tol):
    # ln J of the micro law: the double-float logarithm against CUDA's
    # float64 log of the same (double-float rounded) argument, relative to
    # |ln x|, on a log-uniform grid plus arguments close to 1 (where ln x is
    # small and cancellation would show)
    x = np.exp(np.linspace(np.log(lo), np.log(hi), 200001))
    near1 = 1.0 + np.concatenate([s * 10.0 ** -np.arange(1, 15, 0.25) for s in (1.0, -1.0)])
    x = _df_round(np.concatenate([x, near1]))
    xd = torch.tensor(x, device='cuda')
    out = torch.empty_like(xd)
    rv.rverom_df_log(xd, out)
    ref = torch.log(xd)
    torch.cuda.synchronize()
    err = ((out - ref).abs() / ref.abs().clamp_min(1e-300)).cpu().numpy()
    err[x == 1.0] = np.abs(out.cpu().numpy()[x == 1.0])
    print('max relative error %.3e' % err.max())
    assert err.max() <= tol


def test_peak_probes():
    # every unit reports a throughput of the right order for a GB300
    # (nominal dense rates: FP32 80.5, FP64 1.25, TF32 1125, BF16 2250 TFLOP/s)
    r = {u: rv.rverom_peak_probe(u) for u in ('fp32', 'fp64', 'tf32', 'bf16')}
    print(r)
    assert 40.0 < r['fp32'] < 90.0
    assert 0.4 < r['fp64'] < 1.5
    assert 400.0 < r['tf32'] < 1300.0
    assert 900.0 < r['bf16'] < 2600.0
    assert 1.5 < r['bf16'] / r['tf32'] < 2.5
