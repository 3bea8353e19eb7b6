"""The kernels' size conditions, checked on the host for every geometry a
plan accepts (nx, ny, nz = 8..2048, Nt = 8..4096, window widths 4..16), from
the work split the library itself chooses (nedner_work_split, no device).

Each in-place block FFT needs N * columns <= values per thread * threads;
every chunk must divide its axis; the dynamic shared memory of every kernel
must fit the 227 KB a CTA can have."""
import itertools

import pytest

SMEM_MAX = 227 * 1024
POW2 = [2 ** k for k in range(3, 12)]          # 8 .. 2048
NTS = [2 ** k for k in range(3, 13)]           # 8 .. 4096
WIDTHS = [4, 6, 8, 10, 12, 14, 16]


@pytest.fixture(scope="module")
def nd():
    from paper_1510_01078_gb300 import build as b
    b.build()
    from paper_1510_01078_gb300 import nedner
    return nedner


def check(nx, ny, nz, Nt, s):
    Lx, Ly, Lt = 2 * nx, 2 * ny, 2 * Nt
    bad = []

    def need(cond, what):
        if not cond:
            bad.append(what)

    # spread + x-FFT
    if s["tpl1"] == 2:
        need(s["c1"] == 64 and Nt % 64 == 0, "spread2: 64 time samples per CTA")
        need(s["threads1"] in (256, 512) and s["groups1"] * 32 == s["threads1"], "spread2: one lane group per warp")
        need(Lx * 32 <= 32 * s["threads1"], "spread2: row FFT fits 32 values per thread")
    else:
        need(s["threads1"] == 256 and 2 <= s["c1"] <= 32 and Nt % s["c1"] == 0, "spread: time chunk")
        need(s["groups1"] * s["c1"] == 256, "spread: lane groups fill the CTA")
        need(s["per1"] in (16, 32) and Lx * s["c1"] // 2 <= s["per1"] * 256, "spread: row FFT fits")
    need(s["smem1"] <= SMEM_MAX, "spread: shared memory")
    # split stage (a): block spread over 16-column blocks, x-FFT of nbx complex
    # columns per CTA, chunks of tq samples dividing Nt and the y-FFT's chunk
    if s["split1"]:
        need(Nt >= 64 and Lx >= 64 and (Lx // 16) % s["wpc_s"] == 0, "block spread: whole CTAs of 16-column blocks")
        need(s["tq"] % 64 == 0 and Nt % s["tq"] == 0 and s["tq"] % s["c2f"] == 0, "split: chunk of time samples")
        need(s["tq"] % (2 * s["nbx"]) == 0, "x-FFT: whole CTAs per chunk")
        need(Lx * s["nbx"] == s["perx"] * s["thx"] and s["perx"] in (16, 32) and s["thx"] <= 256, "x-FFT: fits")
        need(s["smem_s"] <= SMEM_MAX and s["smem_x"] <= SMEM_MAX, "split: shared memory")
    # y-FFT (values per thread 16 or 32) and its transpose (16)
    need(Nt % s["c2f"] == 0 and Ly * s["c2f"] <= 16 * 256, "y-FFT: column FFT fits")
    need(s["smem2f"] <= SMEM_MAX, "y-FFT: shared memory")
    # NER and its transpose: line FFT of Lt and z-FFT of nz, 16 values per thread
    need(s["threads3"] in (256, 512) and ny % s["lpc"] == 0, "NER: line groups")
    need(Lt * s["lpc"] <= 16 * s["threads3"] and nz * s["lpc"] <= 16 * s["threads3"], "NER: FFTs fit")
    need(s["smem3"] <= SMEM_MAX and s["smem3a"] <= SMEM_MAX, "NER and its transpose: shared memory")
    # transposed NER: the nz + 1 depth frequencies of a line in chunks of icap3a
    # items (value, first grid point, w + 1 tap-weight slots), all of them (at
    # most 1025) or half where only the half fits four CTAs of 256 per SM
    pad = lambda n: n + (n >> 4)
    base = (pad(Lt * s["lpc"]) + pad(nz * s["lpc"])) * 8
    per_item, four = 8 + 4 + 4 * (s["w"] + 1), 228 * 1024 // 4 - 1024
    need(s["smem3a"] == base + s["icap3a"] * per_item, "transposed NER: items fill the rest")
    all_items, half = min(nz + 1, 1025), (nz + 2) // 2
    if s["icap3a"] == half and half != all_items:
        need(s["threads3"] == 256 and base + all_items * per_item > four >= s["smem3a"],
             "transposed NER: halves only to fit a fourth CTA")
    else:
        need(s["icap3a"] == all_items, "transposed NER: all items, at most 1025")
    # inverse image FFTs and their transposes: 128 threads, 16 values each
    need(nz % s["c4"] == 0 and ny * s["c4"] <= 16 * 128, "y-IFFT: fits")
    need(ny % s["c5"] == 0 and (nx // 2) * s["c5"] <= 16 * 128, "x-c2r: fits")
    need(max(s["smem4"], s["smem5"]) <= SMEM_MAX, "image FFTs: shared memory")
    # transposed gather (adjoint and position gradient)
    if s["tpl_adj"] == 2:
        need(s["ca"] == 64 and Nt % 64 == 0, "gather2: 64 time samples per CTA")
        need(s["threads_adj"] in (256, 512) and Lx * 32 <= 32 * s["threads_adj"], "gather2: row FFT fits")
    else:
        need(2 <= s["ca"] and Nt % s["ca"] == 0, "gather: time chunk")
        need(Lx * s["ca"] // 2 <= s["per_adj"] * 256, "gather: row FFT fits")
    need(s["smem_adj"] <= SMEM_MAX and s["smem_grad"] <= SMEM_MAX, "gather: shared memory")
    return bad


def test_every_accepted_geometry_meets_the_kernel_size_conditions(nd):
    failures = []
    for nx, ny, nz, Nt in itertools.product(POW2, POW2, POW2, NTS):
        for w in WIDTHS:
            s = dict(nd.work_split(nx, ny, nz, Nt, w), w=w)
            bad = check(nx, ny, nz, Nt, s)
            if bad:
                failures.append(((nx, ny, nz, Nt, w), bad))
    assert not failures, failures[:10]


def test_rejected_geometries(nd):
    from paper_1510_01078_gb300.nedner import NednerError
    for args in [(4096, 8, 8, 64, 12), (8, 8, 8, 8192, 12), (12, 8, 8, 64, 12), (8, 8, 8, 64, 3), (8, 8, 8, 64, 18)]:
        with pytest.raises(NednerError):
            nd.work_split(*args)


def test_known_splits(nd):
    """The splits the timed workloads run with."""
    c2 = nd.work_split(128, 128, 256, 512, 12)
    assert (c2["tpl1"], c2["c1"], c2["threads1"], c2["lpc"], c2["tpl_adj"]) == (2, 64, 256, 4, 2)
    c3 = nd.work_split(256, 256, 512, 2048, 12)
    assert (c3["tpl1"], c3["threads1"], c3["lpc"], c3["threads_adj"], c3["c4"], c3["c5"]) == (2, 512, 1, 512, 8, 16)
    assert (c3["split1"], c3["tq"], c3["nbx"], c3["thx"], c3["perx"]) == (1, 2048, 8, 256, 16)
    assert (c2["split1"], c2["nbx"], c2["thx"], c2["perx"]) == (1, 16, 256, 16)
    # the transposed NER holds half of a line's depth frequencies at a time on
    # both (257 of 513 on C3, 55.6 KB; 129 of 257 on C2), for four CTAs per SM
    assert (c3["icap3a"], c3["smem3a"]) == (257, 55616)
    assert (c2["icap3a"], c2["smem3a"]) == (129, 51776)
