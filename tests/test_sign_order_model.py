"""Host-side model of the sign operands' layout and arithmetic (no GPU): the circulant order of the
sample pairs lists every unordered pair once (Algorithm 1's sum is order-free), the packed 16-bit
compares give gt / ge for every rank difference below 5792 without borrowing across lanes, and the
sign-filling byte permute followed by two logic ops yields the FP8 / FP4 / BF16 codes of +1, -1
and 0. The GPU parity tests check the kernels themselves against the oracle."""
import itertools

import numpy as np

M32 = 0xFFFFFFFF


def circulant_pair(k, n):
    d = k // n + 1
    i = k % n
    return i, (i + d) % n


def test_circulant_order_is_a_bijection_onto_pairs():
    for n in list(range(2, 70)) + [127, 128, 129, 255, 256, 301]:
        K = n * (n - 1) // 2
        seen = set()
        for k in range(K):
            i, j = circulant_pair(k, n)
            assert i != j
            p = (min(i, j), max(i, j))
            assert p not in seen
            seen.add(p)
        assert len(seen) == K


def test_packed_compares_have_no_cross_lane_borrow():
    # (a, b) pairs of 16-bit lanes with values below 5792 (the longest contraction rows), both
    # lanes at once, the largest differences included
    vals = np.unique(np.concatenate([np.arange(0, 5792, 13), [1, 5790, 5791]])).astype(np.int64)
    a_lo, b_lo = np.meshgrid(vals, vals[::-1], indexing="ij")
    a_hi, b_hi = b_lo[::-1], a_lo
    A = (a_hi << 16) | a_lo
    B = (b_hi << 16) | b_lo
    G = (B - A + 0x7FFF7FFF) & M32
    E = (B - A + 0x80008000) & M32
    assert np.array_equal((G >> 15) & 1, (b_lo > a_lo).astype(np.int64))
    assert np.array_equal((G >> 31) & 1, (b_hi > a_hi).astype(np.int64))
    assert np.array_equal((E >> 15) & 1, (b_lo >= a_lo).astype(np.int64))
    assert np.array_equal((E >> 31) & 1, (b_hi >= a_hi).astype(np.int64))


def prmt_sign_fill(x, y, sel):
    """prmt.b32 default mode: selector nibble bit 3 replicates the selected byte's sign bit."""
    b = [(x >> (8 * i)) & 0xFF for i in range(4)] + [(y >> (8 * i)) & 0xFF for i in range(4)]
    out = 0
    for i in range(4):
        s = (sel >> (4 * i)) & 0xF
        v = b[s & 7]
        if s & 8:
            v = 0xFF if v & 0x80 else 0
        out |= v << (8 * i)
    return out


def _flags(signs):
    """G, E words for eight signs (+1, -1, 0): lane value b - a = sign."""
    G, E = [], []
    for t in range(4):
        g = e = 0
        for h in range(2):
            s = signs[2 * t + h]
            g |= (0x8000 if s > 0 else 0x7FFF) << (16 * h)
            e |= (0x8000 if s >= 0 else 0x7FFF) << (16 * h)
        G.append(g)
        E.append(e)
    return G, E


def test_operand_codes():
    fp8 = {1: 0x38, -1: 0xB8, 0: 0}
    fp4 = {1: 0x2, -1: 0xA, 0: 0}
    bf16 = {1: 0x3F80, -1: 0xBF80, 0: 0}
    for signs in itertools.product((1, -1, 0), repeat=4):
        signs = list(signs) + list(signs[::-1])
        G, E = _flags(signs)
        # FP8: four bytes per word, elements in order
        for h in range(2):
            mg = prmt_sign_fill(G[2 * h], G[2 * h + 1], 0xFDB9)
            me = prmt_sign_fill(E[2 * h], E[2 * h + 1], 0xFDB9)
            w = ((mg | (~me & M32)) & 0x38383838) | ((~me & M32) & 0x80808080)
            assert [(w >> (8 * i)) & 0xFF for i in range(4)] == [fp8[s] for s in signs[4 * h:4 * h + 4]]
        # FP4: element b in the high nibble of byte b, element 4 + b in the low nibble
        mg0, mg1 = prmt_sign_fill(G[0], G[1], 0xFDB9), prmt_sign_fill(G[2], G[3], 0xFDB9)
        me0, me1 = prmt_sign_fill(E[0], E[1], 0xFDB9), prmt_sign_fill(E[2], E[3], 0xFDB9)
        hg = (mg0 & 0xF0F0F0F0) | (mg1 & 0x0F0F0F0F)
        he = (me0 & 0xF0F0F0F0) | (me1 & 0x0F0F0F0F)
        w = ((hg | (~he & M32)) & 0x22222222) | ((~he & M32) & 0x88888888)
        for b in range(4):
            assert (w >> (8 * b + 4)) & 0xF == fp4[signs[b]]
            assert (w >> (8 * b)) & 0xF == fp4[signs[4 + b]]
        # BF16: two halves per word
        for t in range(4):
            mg = prmt_sign_fill(G[t], G[t], 0xBB99)
            me = prmt_sign_fill(E[t], E[t], 0xBB99)
            w = ((mg | (~me & M32)) & 0x3F803F80) | ((~me & M32) & 0x80008000)
            assert w & 0xFFFF == bf16[signs[2 * t]] and w >> 16 == bf16[signs[2 * t + 1]]


def test_circulant_sign_product_equals_oracle_S():
    """S = A A^T with the signs in circulant order equals the oracle's definition counts on data
    with ties (Algorithm 1's sum does not depend on the order of the sample pairs)."""
    import oracle

    g = np.random.default_rng(4)
    for n in (7, 8, 9, 40):
        X = np.round(g.random((6, n)) * 6) / 6  # heavy ties
        K = n * (n - 1) // 2
        A = np.zeros((6, K), dtype=np.int64)
        for k in range(K):
            i, j = circulant_pair(k, n)
            A[:, k] = np.sign(X[:, j] - X[:, i])
        S = A @ A.T
        for u in range(6):
            for v in range(u + 1, 6):
                assert S[u, v] == oracle.pair_counts(X[u], X[v], "definition")["S"]
