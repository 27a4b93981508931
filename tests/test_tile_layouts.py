"""The tiled kernels' register layouts, read from the library's own index functions on the host
(qvs_tile_layout; no GPU): every layout is a bijection onto its tile, a warp's global access of one
register covers whole 32-byte sectors, and the shared-memory transposes are free of bank conflicts
except where the design says otherwise (column layout 0 at N = 2^25)."""
from collections import defaultdict

import numpy as np
import pytest

import paper_2110_03963_gb300 as qvs

HC, COL, ROW, BOX = (qvs.QVS_LAYOUT_HYPERCUBE, qvs.QVS_LAYOUT_CIRCULANT_COLUMN, qvs.QVS_LAYOUT_CIRCULANT_ROW,
                     qvs.QVS_LAYOUT_CIRCULANT_BOX)


def _wavefronts(slots, lanes_per_phase, words_per_access):
    """Shared-memory wavefronts of one warp instruction: 32 banks of 4 bytes; accesses of
    words_per_access 8-byte words are served lanes_per_phase lanes at a time (16 for 8 bytes,
    8 for 16 bytes), one wavefront per distinct access unit that shares a bank group."""
    groups = 16 // words_per_access
    total = 0
    for p in range(0, len(slots), lanes_per_phase):
        banks = defaultdict(set)
        for s in slots[p:p + lanes_per_phase]:
            unit = s // words_per_access
            banks[unit % groups].add(unit)
        total += max(len(v) for v in banks.values())
    return total


def _ratio(index, slot, lanes_per_phase=16, words=1, regs=None):
    """Wavefronts over the ideal (one per phase) for every warp and register of a layout."""
    T, R = index.shape
    got = ideal = 0
    for r in (range(R) if regs is None else regs):
        for w in range(T // 32):
            got += _wavefronts(slot[index[32 * w:32 * w + 32, r]], lanes_per_phase, words)
            ideal += 32 // lanes_per_phase
    return got / ideal


def _sectors(index, glob, r, words=1):
    """32-byte sectors touched by warp 0's access of register r (words consecutive 8-byte words
    per lane, the first at the register's tile index), and whether every touched sector is full."""
    addr = np.concatenate([glob[index[0:32, r]].astype(np.int64) * 8 + 8 * k for k in range(words)])
    secs = addr // 32
    used = defaultdict(set)
    for a, s in zip(addr.tolist(), secs.tolist()):
        used[s].add(a)
    return len(used), all(len(v) == 4 for v in used.values())


def _bijective(index):
    return sorted(index.ravel().tolist()) == list(range(index.size))


@pytest.mark.parametrize("L", [0, 1, 2, 3])
def test_hypercube_layouts(L):
    index, slot, glob, _ = qvs.qvs_tile_layout(HC, 0, L)
    assert index.shape == (256, 16) and _bijective(index)
    if L == 0:
        # registers 2m, 2m + 1 hold j, j ^ 1 in adjacent, 16-byte aligned slots: one 16-byte access,
        # served 8 lanes at a time; a warp moves 512 contiguous bytes of the state
        assert all(index[t, 2 * m + 1] == index[t, 2 * m] ^ 1 for t in range(256) for m in range(8))
        assert all(slot[j] % 2 == 0 and slot[j ^ 1] == slot[j] + 1 for j in range(0, 4096, 2))
        assert _ratio(index, slot, 8, 2, regs=range(0, 16, 2)) == 1.0
        assert all(_sectors(index, glob, r, 2) == (16, True) for r in range(0, 16, 2))
    else:
        assert _ratio(index, slot) == 1.0
    if L == 2:   # lanes = 32 consecutive tile indices: 256 bytes
        assert all(_sectors(index, glob, r) == (8, True) for r in range(16))
    if L == 3:   # lanes = two runs of 16 consecutive tile indices: two 128-byte rows
        for r in range(16):
            j = np.sort(index[0:32, r])
            assert np.all(np.diff(j[:16]) == 1) and np.all(np.diff(j[16:]) == 1)
            assert _sectors(index, glob, r) == (8, True)


@pytest.mark.parametrize("log2n", list(range(17, 28)))
def test_circulant_column_layouts(log2n):
    ratios = []
    for L in range(3):
        index, slot, glob, cb = qvs.qvs_tile_layout(COL, log2n, L)
        assert index.shape == (512, 32) and _bijective(index)
        ratios.append(_ratio(index, slot))
        if L == 0:
            # the global loads and stores: whole sectors, 8 per warp instruction; at N = 2^27 the
            # tiles are two columns wide, so a lane's row holds 16 bytes and 16 half-used sectors
            for r in range(32):
                n_sec, full = _sectors(index, glob, r)
                assert (n_sec, full) == ((16, False) if log2n == 27 else (8, True)), (log2n, r)
    if log2n == 25:
        # layout 0 at 2 wavefronts per phase: a pass's four transposes (eight accesses, two of them
        # in layout 0) then take 1.25 times the conflict-free count
        assert ratios == [2.0, 1.0, 1.0]
    else:
        assert ratios == [1.0, 1.0, 1.0]


def test_circulant_row_layouts():
    for L in range(3):
        index, slot, glob, _ = qvs.qvs_tile_layout(ROW, 0, L)
        assert index.shape == (512, 32) and _bijective(index)
        assert _ratio(index, slot) == 1.0
    # the row pass loads and stores in layout 2: 256 contiguous bytes per warp instruction
    index, slot, glob, _ = qvs.qvs_tile_layout(ROW, 0, 2)
    assert all(_sectors(index, glob, r) == (8, True) for r in range(32))


def test_tensor_copy_box_at_2_26():
    """The staged column tile of N = 2^26: the box word order is a bijection, and each half-warp's
    layout-0 register lands on 16 consecutive 8-byte words (one 128-byte wavefront)."""
    index, box, _, _ = qvs.qvs_tile_layout(BOX, 26, 0)
    assert sorted(box.tolist()) == list(range(1 << 14))
    for r in range(32):
        for hw in range(32):
            w = np.sort(box[index[16 * hw:16 * hw + 16, r]])
            assert np.all(np.diff(w) == 1) and w[0] % 16 == 0


def test_layout_argument_errors():
    for args in [(HC, 0, 4), (HC, 17, 0), (COL, 16, 0), (COL, 28, 0), (COL, 20, 3), (ROW, 20, 0), (BOX, 25, 0),
                 (BOX, 26, 1), (9, 0, 0)]:
        with pytest.raises(qvs.QvsError):
            qvs.qvs_tile_layout(*args)
