"""Pins of the oracle's random-number layer (reading 8 of the oracle header).

The paper does not say how its normal numbers are drawn, so the counter-based
Philox4x32-10 generator of Salmon et al. (SC'11) is the chosen definition.  The
oracle's implementation is pinned against an independent implementation of the
same published generator: Triton's ``tl.philox``, run by Triton's CPU
interpreter (no GPU is needed).  The uniform and Box-Muller steps are pinned by
their exact and distributional properties.
"""
import json
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
from scipy import stats

from oracle import cmb3d_oracle as orc

TRITON_SCRIPT = textwrap.dedent(r"""
    import os, sys, json
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl

    @triton.jit
    def _k(out_ptr, c_ptr, seed, n, BLOCK: tl.constexpr):
        i = tl.arange(0, BLOCK)
        m = i < n
        c0 = tl.load(c_ptr + 4 * i + 0, mask=m)
        c1 = tl.load(c_ptr + 4 * i + 1, mask=m)
        c2 = tl.load(c_ptr + 4 * i + 2, mask=m)
        c3 = tl.load(c_ptr + 4 * i + 3, mask=m)
        a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
        tl.store(out_ptr + 4 * i + 0, a, mask=m)
        tl.store(out_ptr + 4 * i + 1, b, mask=m)
        tl.store(out_ptr + 4 * i + 2, c, mask=m)
        tl.store(out_ptr + 4 * i + 3, d, mask=m)

    req = json.loads(sys.stdin.read())
    res = []
    for seed, ctrs in req:
        c = torch.tensor(np.array(ctrs, dtype=np.uint32).view(np.int32))
        n = c.numel() // 4
        out = torch.zeros(4 * n, dtype=torch.int32)
        blk = 1 << max(0, (n - 1).bit_length())
        _k[(1,)](out, c, seed, n, BLOCK=blk)
        res.append(out.numpy().view(np.uint32).tolist())
    print(json.dumps(res))
""")


def _triton_philox(requests):
    pytest.importorskip("triton")
    env = dict(os.environ, TRITON_INTERPRET="1")
    p = subprocess.run([sys.executable, "-c", TRITON_SCRIPT], input=json.dumps(requests),
                       capture_output=True, text=True, env=env, timeout=600)
    if p.returncode != 0:
        pytest.skip("Triton CPU interpreter unavailable: " + p.stderr[-300:])
    return json.loads(p.stdout.strip().splitlines()[-1])


def test_philox_matches_independent_implementation():
    rng = np.random.default_rng(12345)
    seeds = [0, 1, 0xFFFFFFFF, 0x123456789ABCDEF0, 0xFFFFFFFFFFFFFFFF, 7 << 32]
    reqs = []
    for s in seeds:
        ctr = rng.integers(0, 2 ** 32, size=(37, 4), dtype=np.uint64)
        ctr[0] = 0
        ctr[1] = 0xFFFFFFFF
        ctr[2] = [5, 17, 300, 0]            # a typical mode counter (m_x, m_y, m_z mod N/2, 0)
        # the triton seed argument is a signed 64-bit integer with the same bits
        sarg = s - (1 << 64) if s >= (1 << 63) else s
        reqs.append((sarg, ctr.tolist()))
    got = _triton_philox(reqs)
    for idx, s in enumerate(seeds):
        ctr = np.array(reqs[idx][1], dtype=np.uint64)
        k0, k1 = orc.seed_key(s)
        w = orc.philox4x32_10(ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3], k0, k1)
        mine = np.stack(w, axis=1).reshape(-1)
        ref = np.array(got[idx], dtype=np.uint64)
        np.testing.assert_array_equal(mine, ref)


def test_philox_zero_block_is_not_identity_and_key_sensitive():
    a = np.stack(orc.philox4x32_10(0, 0, 0, 0, 0, 0))
    b = np.stack(orc.philox4x32_10(0, 0, 0, 0, 1, 0))
    c = np.stack(orc.philox4x32_10(1, 0, 0, 0, 0, 0))
    assert np.all(a != 0)
    assert np.count_nonzero(a != b) == 4 and np.count_nonzero(a != c) == 4


def test_philox_words_are_uniform_bits():
    n = 1 << 16
    w = orc.philox4x32_10(np.arange(n), 3, 9, 0, *orc.seed_key(42))
    bits = np.stack(w).astype(np.uint64)
    # every bit position is set about half the time
    for s in range(32):
        frac = np.mean((bits >> np.uint64(s)) & np.uint64(1))
        assert abs(frac - 0.5) < 5 * 0.5 / np.sqrt(bits.size)


def test_uniform_from_word_exact_range():
    w = np.array([0, 511, 512, 0xFFFFFFFF], dtype=np.uint64)
    u = orc.uniform_from_word(w)
    assert u[0] == 2.0 ** -24 and u[1] == 2.0 ** -24
    assert u[2] == 1.5 * 2.0 ** -23
    assert u[3] == 1.0 - 2.0 ** -24
    # exactly representable in binary32 as well, over the whole range
    w = np.concatenate([w, np.random.default_rng(1).integers(0, 2 ** 32, 100000, dtype=np.uint64)])
    u = orc.uniform_from_word(w)
    assert np.all(u.astype(np.float32).astype(np.float64) == u)
    assert np.all((u > 0) & (u < 1))


def test_box_muller_is_standard_normal():
    n = 1 << 17
    w = orc.philox4x32_10(np.arange(n), 0, 0, 0, *orc.seed_key(7))
    g1, g2 = orc.box_muller(orc.uniform_from_word(w[0]), orc.uniform_from_word(w[1]))
    for g in (g1, g2):
        assert stats.kstest(g, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(g1, g2)[0, 1]) < 5 / np.sqrt(n)
    # closed form at the quarter angle: u1 = 1/4 gives g1 = 0, g2 = sqrt(-2 ln u0)
    a, b = orc.box_muller(np.array([0.5]), np.array([0.25]))
    assert abs(a[0]) < 1e-15 and abs(b[0] - np.sqrt(2 * np.log(2))) < 1e-15
