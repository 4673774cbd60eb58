"""Bank conflicts of the column passes' shared-memory exchanges, modelled on the host.

A host program compiled from the kernel sources prints, for float column
lengths, the plan each kernel uses: elements per thread E (col_E), columns per
tile W (col_W), and for each stage before the last its radix RS, sub-transform
length NS and whether the write and read indices are padded linearly.  A
thread of a tile is (column c, line thread j) = (t mod W, t div W).  The test
replays every exchange's addresses warp by warp and counts shared-memory
wavefronts against the conflict-free count:

* the pipelined kernel (1024 and 2048 points) exchanges real and imaginary
  parts separately through a buffer of 4-byte reals, row r at r + (r >> 5)
  (ColSplitEx): every access must be conflict-free, for 16-column tiles at
  1024 points and for the 8-column tiles of 2048 points;
* the one-tile and one-buffer kernels exchange whole complex values through an
  unpadded [L][W] buffer (ColEx; 8-byte elements, a warp served as two
  half-warps of 128 bytes): with W = 16 every row is one 128-byte segment, so
  every access must be conflict-free as well."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2202_12756_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "kern_impl.cuh"
using namespace fft3d;
template <int L, bool SPLIT> void show()
{
    constexpr int E = col_E<float, L>();
    constexpr int W = col_W<float, L>();
    constexpr int NT = L / E;
    constexpr int P = SPLIT ? ColSplitEx<float, W>::kPadShift : ColEx<float2, W>::kPadShift;
    printf("%d %d %d %d %d %d", L, SPLIT ? 1 : 0, E, W, NT, P);
    for (int s = 0; s + 1 < line_nstages(L, E); ++s) {
        const int rs = line_radix(L, E, s), ns = line_ns(L, E, s);
        printf(" %d,%d,%d,%d", rs, ns, pad_linear<P>(ns, rs) ? 1 : 0, pad_linear_reads<P>(NT) ? 1 : 0);
    }
    printf("\n");
}
int main()
{
    show<1024, true>(); show<2048, true>();
    show<256, false>(); show<512, false>(); show<768, false>(); show<1536, false>();
    return 0;
}
"""


def pad_row(P, lin, base, off):
    if P < 0:
        return base + off
    if lin:
        return base + (base >> P) + off + (off >> P)
    return base + off + ((base + off) >> P)


def wavefronts_4b(addrs):
    """32-bit accesses of one warp: 32 banks of 4 bytes, one wavefront per distinct address in the busiest bank."""
    banks = {}
    for a in set(addrs):
        banks.setdefault(a % 32, set()).add(a)
    return max(len(v) for v in banks.values())


def wavefronts_8b(addrs):
    """64-bit accesses of one warp, served as two half-warps of 16 lanes."""
    total = 0
    for half in (addrs[:16], addrs[16:]):
        banks = {}
        for a in set(half):
            banks.setdefault((2 * a) % 32, set()).add(a)
        total += max(len(v) for v in banks.values())
    return total


def exchange_cost(L, split, E, W, NT, P, stages):
    threads = W * NT
    wf = wavefronts_4b if split else wavefronts_8b
    ideal_per = 1 if split else 2
    got = ideal = 0
    for w0 in range(0, threads, 32):
        lanes = range(w0, w0 + 32)
        for rs, ns, lw, lr in stages:
            for q in range(E // rs):
                for m in range(rs):
                    addrs = []
                    for t in lanes:
                        c, j = t % W, t // W
                        b = j + q * NT
                        base = (b // ns) * ns * rs + (b % ns)
                        addrs.append(pad_row(P, lw, base, m * ns) * W + c)
                    got += wf(addrs)
                    ideal += ideal_per
            for i in range(E):
                got += wf([pad_row(P, lr, t // W, i * NT) * W + t % W for t in lanes])
                ideal += ideal_per
    return got, ideal


@pytest.fixture(scope="module")
def plans(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("colbanks")
    src, exe = d / "cb.cu", d / "cb"
    src.write_text(PROGRAM)
    subprocess.run([nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC,
                    "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True, timeout=600)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60).stdout
    res = {}
    for line in out.strip().splitlines():
        f = line.split()
        L, split, E, W, NT, P = map(int, f[:6])
        res[(L, split)] = (E, W, NT, P, [tuple(map(int, s.split(","))) for s in f[6:]])
    return res


@pytest.mark.parametrize("L", [1024, 2048])
def test_pipelined_split_exchange_conflict_free(plans, L):
    E, W, NT, P, stages = plans[(L, 1)]
    assert (E, P) == (32, 5) and W == (16 if L == 1024 else 8)
    got, ideal = exchange_cost(L, True, E, W, NT, P, stages)
    assert got == ideal, (L, got, ideal)


@pytest.mark.parametrize("L", [256, 512, 768, 1536])
def test_full_width_exchange_conflict_free(plans, L):
    E, W, NT, P, stages = plans[(L, 0)]
    assert W == 16 and P < 0
    got, ideal = exchange_cost(L, False, E, W, NT, P, stages)
    assert got == ideal, (L, got, ideal)
