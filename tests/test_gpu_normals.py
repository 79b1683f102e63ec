"""The thermal normals of Eq. F as the two precisions draw them on the GPU.

Both run one Philox4x64-10 block per particle and step and Box-Muller on two
pairs of 53-bit uniforms.  The FP64 path uses FP64 logarithm, square root and
sine/cosine, so it agrees with the oracle (C library functions) to a few ulp.
The mixed path evaluates the same formulas in double-float arithmetic on the
FP32 pipes (table-driven logarithm and sine/cosine, a Newton-refined square
root); double-float arithmetic keeps about 44 significant bits through the
chain, so its normals agree with the oracle's within 2e-13 max(1, |g|) —
far inside what the mixed path's right-hand side needs (2e-11 of max |b|).
"""
import numpy as np
import pytest

import oracle

ss = pytest.importorskip("paper_1808_06381_gb300")

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed,step", [(20180817, 0), (7, 17), (2**63 + 5, 123456789)])
def test_normals_of_both_precisions_match_the_oracle(seed, step):
    rng = np.random.default_rng(seed % 1000 + step % 1000)
    ids = np.concatenate([np.arange(20000), rng.integers(0, 2**50, 20000)]).astype(np.int64)
    ref = oracle.noise(seed, step, ids)
    g64 = ss.normals(seed, step, ids, "fp64")
    gdf = ss.normals(seed, step, ids, "mixed")
    assert np.all(np.isfinite(gdf))
    assert np.abs(g64 - ref).max() <= 1e-14 * np.maximum(1.0, np.abs(ref)).max()
    assert np.all(np.abs(gdf - ref) <= 2e-13 * np.maximum(1.0, np.abs(ref)))
    # the large-|g| tail (uniforms near 0, logarithms near -37) is covered
    assert np.abs(ref).max() > 4.0


def test_normals_hook_rejects_bad_arguments():
    ids = np.arange(4, dtype=np.int64)
    out = np.zeros((4, 3))
    lib = ss.load()
    assert lib.sp_normals(0, 1, 0, -1, None, 1, None) < 0                       # negative count
    assert lib.sp_normals(0, 1, 0, 4, ids.ctypes.data, 7, out.ctypes.data) < 0   # unknown precision
    assert lib.sp_normals(0, 1, 0, 0, None, 1, None) == 0                        # nothing to do
