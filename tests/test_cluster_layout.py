"""Index arithmetic of the two-CTA 1/128 solve (fem_eval_cluster), restated on the host.

CTA r of a cluster keeps the fine rows 64 r + 1 .. 64 r + 64 of the 1/128 level at local index
(j - 64 r) S + i (S = 130, local rows 0 .. 65 with a halo row on either side), takes the colour
positions [4096 r, 4096 r + 4096) of the red-black enumeration (four red and four black slots per
thread of 1024), sends its boundary row (64 or 65) into the partner's halo at local index
+-64 S, rank 1 sends the red residuals of row 65 (red-only array indexed by n / 2), and the CTAs
restrict the coarse rows 1 .. 32 and 33 .. 63. These tests pin the invariants the kernel relies
on: every interior node in exactly one slot, every value read across the strip boundary is one the
partner sends, the restriction covers every coarse node once and reads only residuals that are
local or sent, and the observation gather finds every node's owner. The GPU parity tests check the
kernel itself against the oracle.
"""
N, T = 128, 1024
S, SC = N + 2, N // 2 + 2
FS = 66 * S


def padded(n):
    return (n + 3) & ~3


def colour_node(k, col):
    """Position k of colour col on level N (G = 16 positions of a row pair per 32)."""
    G = 16
    blk, l = divmod(k, 2 * G)
    R, sg = divmod(blk, N // 2 // G)
    j = 2 * R + 1 + l // G
    i = (1 if ((j & 1) ^ col) else 2) + 2 * (sg * G + l % G)
    return (k < N * N // 2 and j <= N - 1 and i <= N - 1), i, j


def slots():
    """(rank, i, j, local index, red, sends) of every valid slot."""
    out = []
    for rank in (0, 1):
        for tid in range(T):
            for q in range(8):
                red = q < 4
                v, i, j = colour_node(4096 * rank + tid + T * (q if red else q - 4), 0 if red else 1)
                if v:
                    out.append((rank, i, j, (j - 64 * rank) * S + i, red, j == (65 if rank else 64)))
    return out


def test_every_interior_node_in_one_slot_of_its_strip():
    seen = {}
    for rank, i, j, nl, red, _ in slots():
        assert 64 * rank + 1 <= j <= 64 * rank + 64
        assert ((i + j) % 2 == 0) == red
        assert nl - S >= 0 and nl + S < FS and nl < (1 << 14)
        assert (j >> 1) * SC + (i >> 1) < (1 << 13)
        assert (i, j) not in seen
        seen[(i, j)] = rank
    assert len(seen) == (N - 1) ** 2


def test_halo_reads_are_partner_sends():
    sl = slots()
    owner = {(i, j): (r, nl) for r, i, j, nl, _, _ in sl}
    sent = {r: {(i, j): nl for rr, i, j, nl, _, s in sl if rr == r and s} for r in (0, 1)}
    for r in (0, 1):
        shift = 64 * S if r else -64 * S
        for (i, j), nl in sent[r].items():   # the partner's local index of this row
            assert nl + shift == (j - 64 * (1 - r)) * S + i
    for (i, j), (r, _) in owner.items():
        for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            nb = (i + di, j + dj)
            if nb in owner and owner[nb][0] != r:
                assert nb in sent[1 - r]


def test_restriction_covers_coarse_rows_from_local_or_sent_residuals():
    sl = slots()
    owner = {(i, j): (r, nl) for r, i, j, nl, _, _ in sl}
    res_sent = {nl >> 1 for r, i, j, nl, red, s in sl if r == 1 and s and red}
    covered = []
    for rank in (0, 1):
        J0, NJ = (33, 31) if rank else (1, 32)
        for idx in range(NJ * (N // 2 - 1)):
            Jr, I = divmod(idx, N // 2 - 1)
            J, I = J0 + Jr, I + 1
            f = (2 * J - 64 * rank) * S + 2 * I
            for ff, (fi, fj) in ((f, (2 * I, 2 * J)), (f + S + 1, (2 * I + 1, 2 * J + 1)),
                                 (f - S - 1, (2 * I - 1, 2 * J - 1))):
                assert (ff >> 1) < padded(FS // 2)
                if (fi, fj) not in owner:
                    continue   # boundary node: the residual array's zero
                r, nl = owner[(fi, fj)]
                if r == rank:
                    assert nl == ff
                else:   # only rank 0 reads across, row 65, through the sent red residuals
                    assert rank == 0 and fj == 65 and (nl >> 1) + 32 * S == ff >> 1 and (nl >> 1) in res_sent
            covered.append((I, J))
    assert sorted(covered) == sorted((I, J) for I in range(1, N // 2) for J in range(1, N // 2))


def test_observation_gather_finds_each_owner():
    owner = {(i, j): (r, nl) for r, i, j, nl, _, _ in slots()}
    for j in range(N + 1):
        for i in range(N + 1):
            r = 1 if j >= 65 else 0
            nl = (j - 64 * r) * S + i
            assert 0 <= nl < FS
            if (i, j) in owner:
                assert owner[(i, j)] == (r, nl)
