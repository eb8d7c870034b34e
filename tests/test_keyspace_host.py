"""The CUDA path's numbering-scheme functions (key_of / cell_of in
csrc/lbm_internal.cuh, __host__ __device__) compiled as host code with nvcc
and checked without a GPU: keys equal the oracle's bit for bit, and the
inverse used by the assembly walk returns every box cell from its key."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = r'''
#include <cstdio>
#include <cstdlib>
#include "lbm_internal.cuh"
namespace lbm {
int fail(int status, const char*, ...) { return status; }
int cuda_fail(cudaError_t, const char*) { return LBM_ECUDA; }
void clear_error() {}
cudaError_t dev_alloc(void**, size_t, cudaStream_t, bool) { return cudaErrorMemoryAllocation; }
void dev_free(void*, cudaStream_t, bool) {}
}
#include "../csrc/assembly.cu"
int main(int argc, char** argv) {
  int32_t dims[3] = {atoi(argv[1]), atoi(argv[2]), atoi(argv[3])};
  lbm_ordering ord{atoi(argv[4]), {atoi(argv[5]), atoi(argv[6]), atoi(argv[7])}, 0};
  lbm::KeySpace literal, walk;
  if (lbm::make_key_space(dims, ord, false, &literal) || lbm::make_key_space(dims, ord, true, &walk))
    return 2;
  if (argc > 8) {   // sampled cells (xorshift64), for boxes too large to walk
    unsigned long long st = strtoull(argv[9], nullptr, 10) | 1ull;
    for (int s = 0, ns = atoi(argv[8]); s < ns; ++s) {
      int64_t p[3];
      for (int d = 0; d < 3; ++d) {
        st ^= st << 13; st ^= st >> 7; st ^= st << 17;
        p[d] = s < 8 ? ((s >> d) & 1) * (dims[d] - 1) : (int64_t)(st % (unsigned long long)dims[d]);
      }
      const unsigned long long k = lbm::key_of(walk, p[0], p[1], p[2]);
      int64_t a, b, c;
      const bool inside = lbm::cell_of(walk, k, a, b, c);
      printf("%llu %d\n", k, (int)(inside && a == p[0] && b == p[1] && c == p[2]));
    }
    return 0;
  }
  for (int64_t z = 0; z < dims[2]; ++z)
    for (int64_t y = 0; y < dims[1]; ++y)
      for (int64_t x = 0; x < dims[0]; ++x) {
        const unsigned long long k = lbm::key_of(literal, x, y, z);
        int64_t a, b, c;
        const bool inside = lbm::cell_of(walk, lbm::key_of(walk, x, y, z), a, b, c);
        printf("%llu %d\n", k, (int)(inside && a == x && b == y && c == z));
      }
  return 0;
}
'''


@pytest.fixture(scope="module")
def keytool(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("keys")
    src = d / "keys.cu"
    src.write_text(SRC.replace('"../csrc/assembly.cu"',
                               '"' + os.path.join(ROOT, "paper_1111_1129_gb300", "csrc",
                                                  "assembly.cu") + '"'))
    exe = d / "keys"
    subprocess.check_call([nvcc, "-std=c++17", "-O1", "-I" + os.path.join(ROOT, "include"),
                           "-I" + os.path.join(ROOT, "paper_1111_1129_gb300", "csrc"),
                           str(src), "-o", str(exe)])
    return str(exe)


@pytest.mark.parametrize("kind,block", [(0, (1, 1, 1)), (1, (8, 8, 8)), (1, (3, 2, 5)),
                                        (2, (1, 1, 1)), (3, (1, 1, 1)), (4, (1, 1, 1))])
@pytest.mark.parametrize("dims", [(13, 7, 9), (16, 16, 16), (33, 4, 2)])
def test_keys_and_inverse_match_the_oracle(keytool, kind, block, dims):
    out = subprocess.run([keytool, *map(str, dims), str(kind), *map(str, block)],
                         capture_output=True, text=True, check=True).stdout.split()
    keys = np.array(out[0::2], dtype=np.uint64)
    roundtrip = np.array(out[1::2], dtype=int)
    np.testing.assert_array_equal(keys, oracle.keys(kind, dims, block).ravel())
    assert roundtrip.all()


@pytest.mark.parametrize("kind,block", [(0, (1, 1, 1)), (1, (1024, 1024, 1024)), (1, (8, 8, 8))])
def test_inverse_beyond_32_bit_keys(keytool, kind, block):
    """A 1025^3 box (just below 2^31 cells): the inverse takes 32-bit division
    for keys below 2^32 and 64-bit division above.  In 1024^3 blocks the
    key space is 2^33, so the far corner's key is 7 * 2^30; the 8 corners
    and 20,000 seeded cells must come back from their keys.  (The full walk
    of the smaller boxes above pins the keys against the oracle.)"""
    dims = (1025, 1025, 1025)
    out = subprocess.run([keytool, *map(str, dims), str(kind), *map(str, block), "20008", "12345"],
                         capture_output=True, text=True, check=True).stdout.split()
    keys = np.array(out[0::2], dtype=np.uint64)
    assert np.array(out[1::2], dtype=int).all()
    if block[0] == 1024:
        # the plane z = 1024 (4 corners and ~20 sampled cells) lies in the
        # second layer of blocks: keys 4 * 2^30 and up
        assert keys.max() == 7 * 2**30 and (keys >= 2**32).sum() >= 4
    else:
        assert keys.max() < 2**32

