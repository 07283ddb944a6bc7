"""The path kernel's own FP32 Box-Muller pieces (Sec. 3.4; the N(0,1) draws of Eq. 7) against
FP64 references, over every one of the 2^23 uniforms the kernel forms from a Philox word:

- u = (floor(w / 2^9) + 1/2) 2^-23 exactly;
- ln u (the kernel's fitted-polynomial logarithm) within one unit in the last place of the
  FP64 logarithm;
- sqrt(-2 ln u) (a Newton-corrected reciprocal-square-root estimate) equal to the correctly
  rounded square root of the kernel's -2 ln u;
- sin 2 pi u and cos 2 pi u (quadrant reduction and series) within one unit in the last place of
  1 of the FP64 values."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_box_muller_pieces_over_every_uniform():
    import paper_1504_00084_gb300 as S
    k = np.arange(1 << 23, dtype=np.uint32)
    out = S.sdd_debug_unit_math(k << np.uint32(9))
    u, lg, r, sn, cs = (out[:, i] for i in range(5))
    assert np.array_equal(u, ((k.astype(np.float64) + 0.5) * 2.0 ** -23).astype(np.float32))
    u64 = u.astype(np.float64)
    ref = np.log(u64)
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    assert (np.abs(lg.astype(np.float64) - ref) <= ulp).all()
    a = np.float32(-2.0) * lg  # exact: scaling by a power of two
    assert np.array_equal(r, np.sqrt(a))
    one_ulp = 2.0 ** -23
    assert np.abs(sn.astype(np.float64) - np.sin(2 * np.pi * u64)).max() <= one_ulp
    assert np.abs(cs.astype(np.float64) - np.cos(2 * np.pi * u64)).max() <= one_ulp
