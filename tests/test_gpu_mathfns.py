"""The flux kernels' own math routines against CUDA's (through libcgks_diag, which runs the same
device functions the kernels inline, with the same shared-memory coefficient table):

  exp_neg      Tang's table-driven e^x for x <= 0 (32-entry 2^(j/32) table, degree-6 Taylor
               polynomial): within 2 ulp of CUDA's exp on 16.8 million arguments in [-700, 0]
  RegK::rcp    rcp.approx.ftz.f64 refined by two Newton-Raphson steps: bit for bit CUDA's
               correctly rounded __drcp_rn on 4.2 million arguments (both signs, 1e-150..1e150)
  erfc_scaled  erfcx from the piecewise polynomials of cgks_erfcx_table.h times exp_neg(-t^2):
               within 1e-15 relative of CUDA's erfc on [0, 26] (the table's own error is 2e-16
               relative; exp_neg adds 2 ulp; erfc(26) ~ 1e-295 is still normal)

and the FP64 rate the roofline divides by: a DFMA with register operands issues close to 2 per SM
and cycle (1.25 TFLOP/s at 2070 MHz on 152 SMs)."""
import pytest

from paper_2001_01570_gb300 import diag

pytestmark = pytest.mark.gpu


def test_exp_neg_within_2_ulp_of_cuda_exp():
    assert diag.exp_neg_maxulp(1 << 24) <= 2


def test_rcp_is_bitwise_the_correctly_rounded_reciprocal():
    assert diag.rcp_maxulp(1 << 22) == 0


def test_erfc_scaled_matches_cuda_erfc():
    assert diag.erfc_maxrel(1 << 22) <= 1e-15


def test_dfma_register_form_issues_near_two_per_sm_and_cycle():
    r = diag.fp64_rate(0, 4096)
    assert 1.8 <= r["per_sm_cycle"] <= 2.05, r
