"""Launch shapes (threads per key G, value-copy vector width V) against the
CPU oracle.

Every shape the autotuner may pick must give the same results: the probe
group width and the copy vector width change how a row is moved, never
which row or what bytes (Algorithms 1-2 do not depend on them). Each (G, V)
replays the same single-bucket LRU history, filled past lambda 1 so that
phase I runs, on a fresh table: statuses, find rows and masks and the final
state are compared with the oracle bit for bit. Row arrays are also passed
8 bytes and 4 bytes off 16-byte alignment, which leaves 8-byte or 4-byte
vectors as the widest the rows allow."""
import numpy as np
import pytest

import oracle
from paper_2603_17168_gb300 import autotune
from paper_2603_17168_gb300 import workloads as w

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_17168_gb300 as hkv  # noqa: E402
from tests.gpu_util import NAN_BITS, export_state, host, same_state  # noqa: E402


def offset_rows(a: np.ndarray, shift_floats: int):
    """A device float32 [n, dim] tensor holding `a`, whose data starts
    shift_floats floats after a 16-byte aligned address."""
    n, dim = a.shape
    buf = torch.empty(n * dim + 4, dtype=torch.float32, device="cuda")
    v = buf[shift_floats:shift_floats + n * dim].view(n, dim)
    v.copy_(torch.from_numpy(a))
    return v


def replay(nb, dim, g, vec, shift, batches, finds):
    t = hkv.Table(nb * 128, dim, hkv.LRU)
    t.set_launch(g, g)
    t.set_value_vector(vec)
    statuses, rows, masks = [], [], []
    for keys, vals in batches:
        st = torch.empty(keys.size, dtype=torch.uint8, device="cuda")
        t.insert_or_assign(torch.from_numpy(keys.view(np.int64)).cuda(),
                           offset_rows(vals, shift), status_out=st)
        statuses.append(host(st))
    for q in finds:
        out = offset_rows(np.full((q.size, dim), np.uint32(NAN_BITS)).view(np.float32), shift)
        found = torch.empty(q.size, dtype=torch.uint8, device="cuda")
        t.find(torch.from_numpy(q.view(np.int64)).cuda(), out, found)
        torch.cuda.synchronize()
        rows.append(host(out).view(np.uint32).copy())
        masks.append(host(found).astype(bool))
    state = export_state(t)
    t.close()
    return statuses, rows, masks, state


@pytest.mark.parametrize("dim", [32, 30])
def test_every_launch_shape_matches_the_oracle(dim):
    rng = np.random.default_rng(2600 + dim)
    nb = 64
    batches = []
    for _ in range(3):
        keys = w.uniform_keys(rng, 4096, distinct=True)
        batches.append((keys, w.normal_values(rng, keys.size, dim)))
    finds = [np.concatenate([batches[-1][0][:1500], w.uniform_keys(rng, 500)])]
    o = oracle.OracleTable(nb, dim, oracle.LRU)
    ost = [o.insert_or_assign(k, v)[0] for k, v in batches]
    orows, omasks = [], []
    for q in finds:
        ov = np.zeros((q.size, dim), np.uint32)
        ov[:] = NAN_BITS
        r, f, _ = o.find(q, ov.view(np.float32))
        orows.append(r.view(np.uint32))
        omasks.append(f)
    ostate = o.export()
    for g in autotune.CANDIDATES:
        for vec in autotune.VECTORS:
            for shift in (0, 2, 1):
                st, rows, masks, state = replay(nb, dim, g, vec, shift, batches, finds)
                tag = f"G={g} V={vec} shift={shift}"
                for a, b in zip(st, ost):
                    assert np.array_equal(a, b), f"statuses differ ({tag})"
                for a, b, fa, fb in zip(rows, orows, masks, omasks):
                    assert np.array_equal(fa, fb), f"hit masks differ ({tag})"
                    assert np.array_equal(a, b), f"rows differ ({tag})"
                same_state(state, ostate)


def test_tune_picks_and_applies_a_candidate(tmp_path, monkeypatch):
    monkeypatch.setenv("HKV_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    rng = np.random.default_rng(2700)
    nb, dim = 256, 32
    t = hkv.Table(nb * 128, dim, hkv.LRU)
    keys = w.uniform_keys(rng, 16384, distinct=True)
    t.insert_or_assign(torch.from_numpy(keys.view(np.int64)).cuda(),
                       torch.from_numpy(w.normal_values(rng, keys.size, dim)).cuda())
    sample = torch.from_numpy(keys[:8192].view(np.int64)).cuda()
    choice = autotune.tune(t, sample, repeats=1)
    assert choice["find_tpk"] in autotune.CANDIDATES
    assert choice["update_tpk"] in autotune.CANDIDATES
    assert choice["vec_bytes"] in autotune.VECTORS
    assert len(choice["find_ms"]) == len(autotune.CANDIDATES) * len(autotune.VECTORS)
    again = autotune.tune(t, sample, repeats=1)  # from the cache
    assert again["vec_bytes"] == choice["vec_bytes"]
    t.close()
