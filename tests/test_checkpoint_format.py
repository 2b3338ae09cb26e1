"""The checkpoint format without a GPU: a checkpoint built here byte by byte
(with FNV-1a written from its definition) is read back by
icd2s_checkpoint_info, and every kind of damage is refused before any CUDA
call: a flipped payload or checksum byte (ICD2S_ERR_INVARIANT), a short or
long buffer, a wrong magic, version or payload size, nonzero reserved fields,
sizes beyond the library's limits and solution bytes other than 0/1
(ICD2S_ERR_ARG)."""
import struct

import numpy as np
import pytest

from paper_2502_13947_gb300 import build as B
from paper_2502_13947_gb300 import icd2s as I


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def fnv1a64(data: bytes) -> int:
    """FNV-1a, 64-bit: offset basis 14695981039346656037, prime 1099511628211."""
    h = 14695981039346656037
    for byte in data:
        h ^= byte
        h = (h * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def make_blob(n=5, R=3, t_next=7, seed=0xDEADBEEF12345678, best_E=-42, stale=3, version=1, magic=b"ICD2SCKP",
              payload=None, reserved=(0, 0), x=None, seed_rng=0):
    rng = np.random.default_rng(seed_rng)
    if x is None:
        x = rng.integers(0, 2, (R, n), dtype=np.uint8)
    bx = rng.integers(0, 2, n, dtype=np.uint8)
    H = rng.integers(0, 50, (R, n), dtype=np.int32)
    P = 5 * R * n + n if payload is None else payload
    hdr = magic + struct.pack("<IiiiQqiIQQ", version, n, R, t_next, seed, best_E, stale, reserved[0], P,
                              reserved[1])
    assert len(hdr) == 64
    body = hdr + x.tobytes() + bx.tobytes() + H.astype("<i4").tobytes()
    return body + struct.pack("<Q", fnv1a64(body))


def code_of(blob):
    with pytest.raises(I.ICD2SError) as e:
        I.icd2s_checkpoint_info(blob)
    return e.value.code


def test_fnv1a64_small_cases():
    # the empty input is the offset basis; one byte is one xor and one multiply
    assert fnv1a64(b"") == 14695981039346656037
    assert fnv1a64(b"\x00") == (14695981039346656037 * 1099511628211) & 0xFFFFFFFFFFFFFFFF


def test_a_checkpoint_built_from_the_format_is_read_back():
    for n, R, t, seed in [(5, 3, 7, 0xDEADBEEF12345678), (1, 1, 0, 0), (64, 9, 123456, 2 ** 64 - 1)]:
        assert I.icd2s_checkpoint_info(make_blob(n=n, R=R, t_next=t, seed=seed)) == (n, R, t, seed)


def test_damage_is_refused():
    good = make_blob()
    assert I.icd2s_checkpoint_info(good)[0] == 5
    for pos in (64, 64 + 15, 64 + 5 * 3 * 5, len(good) - 9, len(good) - 1, 33):
        bad = bytearray(good)
        bad[pos] ^= 0x01 if 64 <= pos < 64 + 15 + 5 else 0x10  # solution bytes stay 0/1
        assert code_of(bytes(bad)) == I.ERR_INVARIANT, pos
    assert code_of(good[:-1]) == I.ERR_ARG
    assert code_of(good + b"\x00") == I.ERR_ARG
    assert code_of(good[:40]) == I.ERR_ARG
    assert code_of(b"") == I.ERR_ARG
    assert code_of(make_blob(magic=b"ICD2SCKQ")) == I.ERR_ARG
    assert code_of(make_blob(version=2)) == I.ERR_ARG
    assert code_of(make_blob(payload=5 * 3 * 5 + 6)) == I.ERR_ARG
    assert code_of(make_blob(reserved=(1, 0))) == I.ERR_ARG
    assert code_of(make_blob(reserved=(0, 1))) == I.ERR_ARG
    assert code_of(make_blob(n=16385, R=1)) == I.ERR_ARG
    assert code_of(make_blob(t_next=-1)) == I.ERR_ARG
    assert code_of(make_blob(stale=-1)) == I.ERR_ARG
    x = np.zeros((3, 5), np.uint8)
    x[2, 4] = 2
    assert code_of(make_blob(x=x)) == I.ERR_ARG
    assert b"not 0/1" in I.lib().icd2s_last_error()


def test_save_and_restore_check_their_arguments_without_a_gpu():
    L = I.lib()
    assert L.icd2s_state_save(None, 0, None, 0, None) == I.ERR_ARG
    assert L.icd2s_state_restore(None, make_blob(), len(make_blob()), None) == I.ERR_ARG
