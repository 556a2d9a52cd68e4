"""Pins for the oracle's AES-128 (FIPS-197) and its DCF PRG."""
import numpy as np
import pytest

import oracle as O
from conftest import golden


def _kats():
    out = []
    for line in open(golden("fips197_aes128.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, p, c = line.split()
        out.append((bytes.fromhex(k), bytes.fromhex(p), bytes.fromhex(c)))
    return out


@pytest.mark.parametrize("key,pt,ct", _kats())
def test_fips197_known_answers(key, pt, ct):
    assert O.aes128(key, pt) == ct


def test_sbox_definition_points():
    # FIPS-197 Sec. 5.1.1: S(0x53) = 0xED; the affine constant gives S(0) = 0x63.
    assert O.sbox(0x53) == 0xED
    assert O.sbox(0x00) == 0x63
    # the S-box is a permutation with no fixed points and no opposite fixed points
    vals = [O.sbox(x) for x in range(256)]
    assert sorted(vals) == list(range(256))
    assert all(v != x and v != (x ^ 0xFF) for x, v in enumerate(vals))


def test_aes_matches_openssl_on_random_blocks():
    """Cross-check against an independent implementation (OpenSSL via the
    cryptography package); used only here, never linked into the oracle."""
    cr = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    rng = np.random.default_rng(11)
    for _ in range(200):
        key = rng.bytes(16)
        blk = rng.bytes(16)
        enc = cr.Cipher(cr.algorithms.AES(key), cr.modes.ECB()).encryptor()
        assert O.aes128(key, blk) == enc.update(blk) + enc.finalize()


def test_mmo_is_tweaked_matyas_meyer_oseas():
    """H(s, j) = AES_K(s ^ j) ^ s ^ j with K = "FuseFSS-DCF-AES!" and j XORed
    into the low 32 bits (little endian); checked against OpenSSL."""
    cr = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    K = b"FuseFSS-DCF-AES!"
    rng = np.random.default_rng(12)
    for j in [0, 1, 2, 3, 5, 0xDEADBEEF]:
        s = rng.bytes(16)
        inp = bytearray(s)
        for i in range(4):
            inp[i] ^= (j >> (8 * i)) & 0xFF
        enc = cr.Cipher(cr.algorithms.AES(K), cr.modes.ECB()).encryptor()
        a = enc.update(bytes(inp)) + enc.finalize()
        expect = bytes(x ^ y for x, y in zip(a, inp))
        assert O.mmo(s, j) == expect
