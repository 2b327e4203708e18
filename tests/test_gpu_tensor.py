"""The library's tcgen05 tensor-core path on the GB300 (sm_103a): a BF16 x BF16
-> FP32 product through shared-memory descriptors and tensor memory, checked
bit for bit against the exact integer product."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_08981_gb300 import build as b
    b.build()
    import paper_2412_08981_gb300 as pkg
    pkg.load()
    return pkg


def test_tcgen05_product_is_exact(P):
    assert P.msp.tensor_selftest() == 0
    # a second run on the same device (tensor memory freed by the first)
    assert P.msp.tensor_selftest() == 0
