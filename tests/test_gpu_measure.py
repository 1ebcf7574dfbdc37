"""The random-access measurement hook: rates are positive and ordered as the
memory system orders them (an 8-byte access costs a whole sector, so it is no
faster than a 32-byte one, and a 128-byte line costs about as much), and the
useful bandwidth of line reads stays below the sequential copy peak."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_17168_gb300 as hkv  # noqa: E402


def test_random_access_rates_are_ordered():
    buf = 2 << 30  # 2 GiB: far above L2
    n = 16 << 20
    line = hkv.measure_random_access(128, buffer_bytes=buf, accesses=n, repeats=2)
    sector = hkv.measure_random_access(32, buffer_bytes=buf, accesses=n, repeats=2)
    word = hkv.measure_random_access(8, buffer_bytes=buf, accesses=n, repeats=2)
    wline = hkv.measure_random_access(128, write=True, buffer_bytes=buf, accesses=n, repeats=2)
    for r in (line, sector, word, wline):
        assert 1e8 < r < 1e12
    assert word < 1.5 * sector
    assert line < sector * 1.5
    assert line * 128 < 10e12  # below any HBM3e sequential rate
