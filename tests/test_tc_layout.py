"""The tensor-core gate's operand layout and descriptors, on the host (no
GPU): the header's layout function is compiled with the host compiler and
checked to place every element of a 128 x 32 BF16 tile at its own in-bounds,
aligned byte (so the MMA operands the tcgen05 gate kernel writes fill their
8 KB tiles exactly), with core matrices of 8 rows x 16 bytes whose neighbours
along K and along the rows lie at the descriptor's two byte offsets, and the
descriptors' fields decode back to the layout and shape the kernel uses."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2306_04467_gb300", "csrc")

PROG = r'''
#include <cstdio>
#include "tcgen05.cuh"
using namespace gks2l::tc;
int main() {
  for (unsigned r = 0; r < 128; r++)
    for (unsigned k = 0; k < 32; k++) printf("%u\n", tile_offset(r, k));
  printf("D %llu\n", (unsigned long long)smem_desc(0x1230));
  printf("I %u\n", idesc_bf16(128, 32));
  return 0;
}
'''


@pytest.fixture(scope="module")
def out(tmp_path_factory):
    d = tmp_path_factory.mktemp("tc")
    src, exe = d / "t.cpp", d / "t"
    src.write_text(PROG)
    subprocess.check_call(["g++", "-std=c++17", "-D__host__=", "-D__device__=", "-I", CSRC, str(src), "-o", str(exe)])
    return subprocess.check_output([str(exe)], text=True).split("\n")


def test_tile_layout_is_a_packing_of_core_matrices(out):
    offs = [int(x) for x in out[:128 * 32]]
    assert sorted(offs) == list(range(0, 8192, 2))          # every BF16 slot of the 8 KB tile, once
    off = lambda r, k: offs[r * 32 + k]
    for r in range(128):
        for k in range(32):
            g, c = r // 8, k // 8
            base = off(8 * g, 8 * c)
            assert off(r, k) == base + (r % 8) * 16 + (k % 8) * 2   # 8 rows of 16 contiguous bytes
            assert base == g * 512 + c * 128                          # SBO along rows, LBO along K


def test_descriptors_decode_to_the_layout_and_shape(out):
    desc = int(next(x for x in out if x.startswith("D ")).split()[1])
    assert desc & 0x3FFF == 0x1230 >> 4                       # start address / 16
    assert (desc >> 16) & 0x3FFF == 128 >> 4                  # leading (K) byte offset / 16
    assert (desc >> 32) & 0x3FFF == 512 >> 4                  # stride (row) byte offset / 16
    assert (desc >> 46) & 0x3 == 1 and desc >> 61 == 0        # descriptor version 1, no swizzle
    idesc = int(next(x for x in out if x.startswith("I ")).split()[1])
    assert (idesc >> 4) & 3 == 1                              # FP32 accumulator
    assert (idesc >> 7) & 7 == 1 and (idesc >> 10) & 7 == 1   # BF16 A and B
    assert (idesc >> 15) & 3 == 0                             # both K-major
    assert (idesc >> 17) & 0x3F == 32 >> 3 and (idesc >> 24) & 0x1F == 128 >> 4
