"""L2 residency of the digest array: turning the window on and off never
changes results (find and upsert on a table with the window give the same
statuses, rows and final state as on a twin without it)."""
import numpy as np
import pytest

from paper_2603_17168_gb300 import workloads as w

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_17168_gb300 as hkv  # noqa: E402
from tests.gpu_util import dev, export_state, host, same_state  # noqa: E402


def test_l2_window_changes_no_result():
    rng = np.random.default_rng(9300)
    a = hkv.Table(256 * 128, 16, hkv.LFU)
    b = hkv.Table(256 * 128, 16, hkv.LFU)
    assert a.l2_residency == 0
    a.set_l2_residency(1 << 40)  # capped at the digest array
    assert a.l2_residency in (0, 256 * 128)  # 0 where the device has no persisting L2
    z = w.Zipf(1.05, 60000)
    for r in range(6):
        keys = dev(z.keys(rng, 8000))
        vals = dev(w.normal_values(rng, 8000, 16))
        sa = torch.empty(8000, dtype=torch.uint8, device="cuda")
        sb = torch.empty(8000, dtype=torch.uint8, device="cuda")
        a.insert_or_assign(keys, vals, status_out=sa)
        b.insert_or_assign(keys, vals, status_out=sb)
        fa = torch.zeros((8000, 16), device="cuda")
        fb = torch.zeros((8000, 16), device="cuda")
        a.find(keys, fa)
        b.find(keys, fb)
        torch.cuda.synchronize()
        assert np.array_equal(host(sa), host(sb))
        assert np.array_equal(host(fa).view(np.uint32), host(fb).view(np.uint32))
        if r == 3:
            a.set_l2_residency(0)
            assert a.l2_residency == 0
    same_state(export_state(a), export_state(b))
