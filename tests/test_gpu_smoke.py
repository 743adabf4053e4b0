"""The round-end smoke entry point itself: one small FP64 step sequence against the oracle,
then the split form with radiation, on cuda:0."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)


def test_smoke_entry_point():
    import __graft_entry__
    __graft_entry__.smoke()
