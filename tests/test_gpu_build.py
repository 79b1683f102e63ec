"""The GPU runs this library's device code as built for sm_103a (no JIT from another target)."""
import pytest

ss = pytest.importorskip("paper_1808_06381_gb300")

pytestmark = pytest.mark.gpu


def test_device_code_is_sm_103():
    binary, ptx = ss.device_code_version(0)
    assert binary == 103, binary
    assert ptx == 103, ptx
