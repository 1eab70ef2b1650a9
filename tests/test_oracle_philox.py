"""Pins of the oracle's core engine (Philox4x32-10) and its counter layout.

The independent pin is the Philox4x32-10 function of the CUDA toolkit's
cuRAND *source header*, compiled here for the host (nvcc, no GPU needed) and
fed the same (counter, key) pairs.  A plain Python-int restatement is a second
check.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

HOST_SRC = r"""
#define QUALIFIERS static inline __host__ __device__
#include <cstdio>
#include <cstdint>
#include <curand_philox4x32_x.h>
int main() {
  unsigned int in[6];
  while (fread(in, sizeof(unsigned int), 6, stdin) == 6) {
    uint4 c = make_uint4(in[0], in[1], in[2], in[3]);
    uint2 k = make_uint2(in[4], in[5]);
    uint4 r = curand_Philox4x32_10(c, k);
    unsigned int out[4] = {r.x, r.y, r.z, r.w};
    fwrite(out, sizeof(unsigned int), 4, stdout);
  }
  return 0;
}
"""


def _nvcc():
    for p in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if p and os.path.exists(p):
            return p
    return None


@pytest.fixture(scope="module")
def curand_host():
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    d = tempfile.mkdtemp(prefix="philox_host_")
    src = os.path.join(d, "p.cu")
    exe = os.path.join(d, "p")
    with open(src, "w") as f:
        f.write(HOST_SRC)
    subprocess.run([nvcc, "-O1", "-o", exe, src], check=True, capture_output=True)
    yield exe
    shutil.rmtree(d, ignore_errors=True)


def _cases(n, seed=7):
    rng = np.random.default_rng(seed)
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    # structured cases: zeros, all-ones, small counters
    ctr[0] = 0
    key[0] = 0
    ctr[1] = 0xFFFFFFFF
    key[1] = 0xFFFFFFFF
    ctr[2] = [1, 0, 0, 0]
    ctr[3] = [0, 0, 0, 1]
    return ctr, key


def test_philox_matches_curand_header(oracle, curand_host):
    ctr, key = _cases(20000)
    inp = np.concatenate([ctr, key], axis=1).astype(np.uint32).tobytes()
    res = subprocess.run([curand_host], input=inp, capture_output=True, check=True)
    want = np.frombuffer(res.stdout, dtype=np.uint32).reshape(-1, 4)
    got = np.stack([oracle.philox4x32_10(c, k) for c, k in zip(ctr, key)])
    assert want.shape == got.shape
    assert np.array_equal(want, got)


def _philox_py(ctr, key):
    M0, M1, W0, W1 = 0xD2511F53, 0xCD9E8D57, 0x9E3779B9, 0xBB67AE85
    c = [int(x) for x in ctr]
    k0, k1 = int(key[0]), int(key[1])
    for r in range(10):
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        c = [(p1 >> 32) ^ c[1] ^ k0, p1 & 0xFFFFFFFF, (p0 >> 32) ^ c[3] ^ k1, p0 & 0xFFFFFFFF]
        k0 = (k0 + W0) & 0xFFFFFFFF
        k1 = (k1 + W1) & 0xFFFFFFFF
    return c


def test_philox_python_restatement(oracle):
    ctr, key = _cases(2000, seed=11)
    for c, k in zip(ctr, key):
        assert list(oracle.philox4x32_10(c, k)) == _philox_py(c, k)


@pytest.mark.parametrize("domain", [0, 1, 2, 3, 4])
def test_counter_layout(oracle, domain):
    seed = 0x0123456789ABCDEF
    stream = 77
    first_block = (5 << 32) + 3  # crosses into the high counter word
    words = oracle.philox_words(seed, domain, stream, first_block, 3)
    for b in range(3):
        blk = first_block + b
        ctr = [blk & 0xFFFFFFFF, domain, stream, blk >> 32]
        key = [seed & 0xFFFFFFFF, seed >> 32]
        assert list(words[4 * b:4 * b + 4]) == _philox_py(ctr, key)


def test_element_words_follow_block_slots(oracle):
    seed, stream = 42, 9
    for dom in (0, 1, 2):
        _, w = oracle.elements(seed, dom, stream, 0, 16)
        ref = oracle.philox_words(seed, dom, stream, 0, 4)
        assert np.array_equal(w, ref)
    # U64: element j owns words 2(j%2), 2(j%2)+1 of block j/2
    _, w = oracle.elements(seed, 4, stream, 0, 8)
    ref = oracle.philox_words(seed, 4, stream, 0, 4)
    assert np.array_equal(w, ref[0::2])


def test_word_bits_balanced(oracle):
    w = oracle.philox_words(42, 0, 0, 0, 1 << 16)
    bits = np.unpackbits(w.view(np.uint8)).reshape(-1, 32).mean(axis=0)
    # each of the 32 bit positions is set half the time (n = 2^18 words)
    assert np.all(np.abs(bits - 0.5) < 5 * 0.5 / np.sqrt(w.size))
