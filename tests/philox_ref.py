"""Philox4x32-10 in plain Python (Salmon et al., SC'11), used by the tests
to re-derive random choices independently of both implementations."""

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    c0, c1, c2, c3 = [int(v) & MASK for v in ctr]
    k0, k1 = [int(v) & MASK for v in key]
    for r in range(10):
        if r:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0
        p1 = M1 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0) & MASK, p1 & MASK, ((p0 >> 32) ^ c3 ^ k1) & MASK, p0 & MASK
    return c0, c1, c2, c3


def below(u, n):
    return (int(u) * int(n)) >> 32


def key_of(seed):
    return (seed & MASK, (seed >> 32) & MASK)
