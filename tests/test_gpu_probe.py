"""The L2 micro-benchmark behind the memory side of the roofline reads what it
claims to read: the coalesced read touches every word of the buffer, and the
gather visits the words its index hash names (checked against the same hash
evaluated with numpy on the host)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fvv():
    from paper_1903_11785_gb300.build import build
    build()
    from paper_1903_11785_gb300 import fvv as mod
    return mod


def _hash(t, i, mask):
    x = t * np.uint32(0x9E3779B9) + np.full_like(t, i) * np.uint32(0x85EBCA6B)
    x ^= x >> np.uint32(16)
    x = x * np.uint32(0x7FEB352D)
    x ^= x >> np.uint32(15)
    return x & np.uint32(mask)


def test_read_probe_touches_every_word(fvv):
    g = torch.Generator(device="cuda").manual_seed(5)
    buf = torch.randint(-2 ** 31, 2 ** 31 - 1, (1 << 16,), dtype=torch.int32, device="cuda", generator=g)
    blocks, threads = 7, 96          # ragged: 672 threads over 16384 chunks of 16 bytes
    out = torch.empty(blocks * threads, dtype=torch.int32, device="cuda")
    fvv.fvv_probe_l2(0, buf, 3, out, blocks, threads)
    torch.cuda.synchronize()
    want = np.bitwise_xor.reduce(buf.cpu().numpy().view(np.uint32))
    assert np.bitwise_xor.reduce(out.cpu().numpy().view(np.uint32)) == want
    fvv.fvv_probe_l2(0, buf, 2, out, blocks, threads)    # every word twice: all zero
    torch.cuda.synchronize()
    assert not out.any()


def test_gather_probe_follows_its_hash(fvv):
    g = torch.Generator(device="cuda").manual_seed(6)
    words = 1 << 12
    buf = torch.randint(-2 ** 31, 2 ** 31 - 1, (words,), dtype=torch.int32, device="cuda", generator=g)
    blocks, threads, reps = 3, 64, 7   # 7 = one group of 4 and a tail of 3
    out = torch.empty(blocks * threads, dtype=torch.int32, device="cuda")
    fvv.fvv_probe_l2(1, buf, reps, out, blocks, threads)
    torch.cuda.synchronize()
    host = buf.cpu().numpy().view(np.uint32)
    t = np.arange(blocks * threads, dtype=np.uint32)
    want = np.zeros_like(t)
    for i in range(reps):
        want ^= host[_hash(t, i, words - 1)]
    assert np.array_equal(out.cpu().numpy().view(np.uint32), want)


def test_probe_rejects_bad_arguments(fvv):
    buf = torch.zeros(100, dtype=torch.int32, device="cuda")      # 400 bytes: not a power of two
    out = torch.empty(256, dtype=torch.int32, device="cuda")
    with pytest.raises(fvv.FvvError):
        fvv.fvv_probe_l2(1, buf, 1, out, 1, 256)
    with pytest.raises(fvv.FvvError):
        fvv.fvv_probe_l2(2, buf, 1, out, 1, 256)
    with pytest.raises(fvv.FvvError):
        fvv.fvv_probe_l2(0, buf, 1, out, 1, 48)                    # threads not a multiple of 32


def test_fma_probe_computes_its_chains(fvv):
    """With a = 1 and b = 0.5 every chain adds 0.5 per step, exactly (small
    binary32 values): thread t's sum is the sum over chains k of
    ((t + k) mod 8) + reps / 2."""
    blocks, threads, reps = 5, 96, 37
    out = torch.empty(blocks * threads, dtype=torch.float32, device="cuda")
    fvv.fvv_probe_fma(reps, 1.0, 0.5, out, blocks, threads)
    torch.cuda.synchronize()
    t = np.arange(blocks * threads)
    want = sum(((t + k) % 8) + reps * 0.5 for k in range(16))
    assert np.array_equal(out.cpu().numpy(), want.astype(np.float32))
    with pytest.raises(fvv.FvvError):
        fvv.fvv_probe_fma(0, 1.0, 0.5, out, blocks, threads)
