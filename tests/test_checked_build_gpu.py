"""The checked build (every indexed load and store of the kernels tested against its
array, a failure recorded in the device error word instead of a fault) runs the library's
kernel families without a single out-of-range index, and gives the default build's
results bit for bit (the adjoint's FP64 atomic sums to rounding). It stands in for a
memory checker, which this pool does not offer; the checked library is loaded in a child
process of its own."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0912_3223_gb300 import build
    build.build()
    build.build(checked=True)


def test_checked_build_is_clean_and_identical(tmp_path):
    out = str(tmp_path / "checked.npz")
    code = ("import sys; sys.path[:0] = [%r, %r]; import numpy as np; import checked_cases; "
            "np.savez(%r, **checked_cases.run_cases())" % (HERE, ROOT, out))
    env = dict(os.environ, LPM_CHECKED_BUILD="1")
    run = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=900)
    # an index outside its array surfaces as LPM_E_CUDA ("a grid index fell outside its
    # array") from the first read-back after it
    assert run.returncode == 0, run.stderr[-3000:]
    import checked_cases
    ref = checked_cases.run_cases()
    got = np.load(out)
    assert sorted(got.files) == sorted(ref)
    for k, v in ref.items():
        if k.startswith("adj_"):
            # receptor sums and gradients are FP64 atomic sums over particles, whose order
            # changes from run to run
            np.testing.assert_allclose(got[k], v, rtol=1e-12, atol=1e-300, err_msg=k)
        else:
            assert np.array_equal(got[k], v), k
