"""Pin the oracle's Philox4x32-10 against a library routine (Triton's philox, CPU interpreter)."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from oracle import philox

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_SCRIPT = textwrap.dedent(r"""
    import os, sys
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl

    @triton.jit
    def k(c_ptr, out_ptr, seed, N: tl.constexpr):
        off = tl.arange(0, N)
        c0 = tl.load(c_ptr + off * 4 + 0).to(tl.uint32)
        c1 = tl.load(c_ptr + off * 4 + 1).to(tl.uint32)
        c2 = tl.load(c_ptr + off * 4 + 2).to(tl.uint32)
        c3 = tl.load(c_ptr + off * 4 + 3).to(tl.uint32)
        r0, r1, r2, r3 = tl.philox(seed, c0, c1, c2, c3)
        tl.store(out_ptr + off * 4 + 0, r0)
        tl.store(out_ptr + off * 4 + 1, r1)
        tl.store(out_ptr + off * 4 + 2, r2)
        tl.store(out_ptr + off * 4 + 3, r3)

    ctr = np.load(sys.argv[1])
    seed = int(sys.argv[2])
    c = torch.from_numpy(ctr.astype(np.uint32).view(np.int32).copy())
    out = torch.zeros(ctr.size, dtype=torch.int32)
    k[(1,)](c, out, seed, N=ctr.shape[0])
    np.save(sys.argv[3], out.numpy().view(np.uint32))
""")


def _triton_available():
    try:
        import triton  # noqa: F401
        return True
    except Exception:
        return False


@pytest.mark.skipif(not _triton_available(), reason="triton not importable")
@pytest.mark.parametrize("seed", [0, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_triton(tmp_path, seed):
    rng = np.random.default_rng(7)
    ctr = rng.integers(0, 2 ** 32, size=(64, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    np.save(tmp_path / "c.npy", ctr)
    script = tmp_path / "t.py"
    script.write_text(_SCRIPT)
    subprocess.run([sys.executable, str(script), str(tmp_path / "c.npy"), str(seed),
                    str(tmp_path / "o.npy")], check=True, cwd=ROOT, timeout=600)
    ref = np.load(tmp_path / "o.npy").reshape(64, 4)
    got = philox.philox4x32_10(ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3],
                               seed & 0xFFFFFFFF, seed >> 32)
    got = np.stack(got, axis=1)
    assert np.array_equal(got, ref)


def test_uniform_range_and_exactness():
    w = np.array([0, 1, 511, 512, 0xFFFFFFFF, 0x80000000], dtype=np.uint32)
    u = philox.words_to_uniform(w)
    assert np.all(u > 0) and np.all(u < 1)
    assert np.array_equal(u.astype(np.float32).astype(np.float64), u)
    assert u[0] == 2.0 ** -24 and u[4] == 1.0 - 2.0 ** -24


def test_stream_layout_blocks():
    # words 4..7 of a sample come from block 1 of the same counter
    w = philox.stream_words(5, 3, 7, np.array([11, 2 ** 33 + 1]), 8)
    r = philox.philox4x32_10(np.array([11, 1]), np.array([0, 2]), 3, (7 << 8) | 1, 5, 0)
    assert np.array_equal(w[4:8], np.stack(r))
