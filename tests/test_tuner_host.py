"""Host logic of the launch-shape autotuner on CPU: every candidate shape lies
in the ranges the C ABI documents for its parity and variant, the per-domain
filter drops exactly the shapes a domain refuses (bulk-staged BF16; the
moment-space operators beyond their variants and 2 cells; the even variant 5
of the moment-space operators for SRT/TRT), and the JSON cache round-trips."""
import pytest

from paper_2408_06880_gb300 import _capi as A
from paper_2408_06880_gb300 import tuner as T


def _documented(parity, shape):
    threads, cells, variant = shape
    warp_multiple = 32 <= threads <= 256 and threads % 32 == 0
    if parity == 0:
        if variant == 0:
            return warp_multiple and cells in (1, 2, 4)
        if variant in (1, 3):
            return threads in (64, 128) and cells in (2, 4)
        if variant == 2:
            return warp_multiple and cells in (2, 4)
        if variant == 5:
            return threads == 128 and cells == 1
        return False
    if variant == 0:
        return warp_multiple and cells in (1, 2)
    if variant == 1:
        return threads in (64, 128) and cells in (2, 4)
    if variant in (2, 4):
        return warp_multiple and cells in (1, 2)
    if variant in (3, 5):
        return warp_multiple and cells == 1
    return False


def test_every_candidate_is_a_documented_shape():
    for s in T.EVEN_SHAPES:
        assert _documented(0, s), s
    for s in T.ODD_SHAPES:
        assert _documented(1, s), s
    assert len(set(T.EVEN_SHAPES)) == len(T.EVEN_SHAPES)
    assert len(set(T.ODD_SHAPES)) == len(T.ODD_SHAPES)


def _info(op=A.TRT, storage=A.FP32, links=0):
    return {"op": op, "storage": storage, "n_bc_links": links}


@pytest.mark.parametrize("storage", [A.FP32, A.FP16])
def test_srt_trt_domains_take_every_candidate(storage):
    for op in (A.SRT, A.TRT):
        # even variant 5 is the moment-space operators' register-bounded kernel
        assert all(T._valid(_info(op, storage), 0, s) == (s[2] != 5) for s in T.EVEN_SHAPES)
        assert all(T._valid(_info(op, storage), 1, s) for s in T.ODD_SHAPES)


def test_bf16_drops_only_the_bulk_staged_shapes():
    info = _info(A.TRT, A.BF16)
    dropped_even = [s for s in T.EVEN_SHAPES if not T._valid(info, 0, s)]
    dropped_odd = [s for s in T.ODD_SHAPES if not T._valid(info, 1, s)]
    assert dropped_even and all(s[2] in (1, 3, 5) for s in dropped_even)
    assert all(s[2] == 1 for s in dropped_odd)
    # odd variant 3 (slots re-read) is not staged: BF16 keeps it
    assert T._valid(info, 1, (128, 1, 3))


@pytest.mark.parametrize("op", [A.MRT, A.CM, A.CUMULANT])
@pytest.mark.parametrize("links", [0, 5])
def test_moment_operators_keep_their_variants(op, links):
    info = _info(op, A.FP32, links)
    for parity, shapes in ((0, T.EVEN_SHAPES), (1, T.ODD_SHAPES)):
        for s in shapes:
            if s[2] == 5:
                want = tuple(s[:2]) == (128, 1)
            elif parity == 0:
                want = s[1] <= 2 and (s[2] == 0 or (op == A.MRT and s[2] == 2))
            else:
                want = s[1] <= 2 and (s[2] in (0, 2) or (s[2] == 3 and links == 0))
            assert T._valid(info, parity, s) == want, (parity, s)


def test_size_class_is_the_log2_bucket():
    assert T.size_class(1) == 0 and T.size_class(0) == 0
    assert T.size_class(1023) == 9 and T.size_class(1024) == 10
    assert T.size_class(8_388_390) == 22


def test_cache_round_trip(monkeypatch, tmp_path):
    path = tmp_path / "sub" / "tune.json"
    monkeypatch.setenv("SLBM_TUNE_CACHE", str(path))
    assert T.cache_path() == str(path)
    assert T._load() == {}
    T._store({"gpu|q19|op1|st0|n22|p0": {"shape": [64, 4, 2], "ms": 0.186}})
    assert T._load()["gpu|q19|op1|st0|n22|p0"]["shape"] == [64, 4, 2]
    assert [p.name for p in path.parent.iterdir()] == ["tune.json"]     # no temporary left behind
