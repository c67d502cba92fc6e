"""Half-byte symbol counting of Sec. 3 (Fig. 2, Sec. 3.1-3.2), restated on Python integers.

TEST INFRASTRUCTURE ONLY: a second, independent way to count one symbol in a 2-bit packed
BWT word, used to cross-check the oracle's plain scan and pinned by the intermediate words
that Fig. 2 prints.  It is written from the prose of Sec. 3 (lookup of both nibbles of each
byte, complemented low table, shift of the wanted 2-bit counter to the bottom of each byte,
fill/mask, sum of absolute byte differences), not from any instruction listing.

Packing: symbol j of a 64-bit word sits at bits 2j..2j+1 (little-endian), codes A=0 C=1 G=2
T=3.  A byte-table entry holds, for the two symbols of a nibble, four 2-bit counters with
counter X at bits 2X..2X+1.
"""
from __future__ import annotations

_FILL = 0xFCFCFCFCFCFCFCFC
_LOW2 = 0x0303030303030303


def pack(codes) -> int:
    w = 0
    for j, c in enumerate(codes):
        w |= (int(c) & 3) << (2 * j)
    return w


def nibble_tables():
    """Lookup tables of Sec. 3.1: per nibble value, the four 2-bit counters packed in a byte;
    the low-nibble table is stored complemented."""
    lo, hi = [], []
    for v in range(16):
        cnt = [0, 0, 0, 0]
        cnt[v & 3] += 1
        cnt[v >> 2] += 1
        byte = sum(cnt[x] << (2 * x) for x in range(4))
        lo.append(~byte & 0xFF)
        hi.append(byte)
    return lo, hi


def _bytes_to_word(bs) -> int:
    return int.from_bytes(bytes(bs), "little")


def count_in_word(word: int, x: int, trace: dict | None = None) -> int:
    """Occurrences of symbol x among the 32 symbols of ``word`` (Sec. 3.1-3.2)."""
    lo_t, hi_t = nibble_tables()
    b = word.to_bytes(8, "little")
    lo_n = [v & 15 for v in b]
    hi_n = [v >> 4 for v in b]
    lo_l = _bytes_to_word(lo_t[v] for v in lo_n)
    hi_l = _bytes_to_word(hi_t[v] for v in hi_n)
    lo_s = lo_l >> (2 * x)                 # counter X to the low two bits of every byte
    hi_s = hi_l >> (2 * x)
    lo_f = lo_s | _FILL                    # Lo: high six bits set -> bytes hold 255 - lo_X
    hi_m = hi_s & _LOW2                    # Hi: high six bits cleared -> bytes hold hi_X
    sad = sum(abs(((lo_f >> (8 * j)) & 255) - ((hi_m >> (8 * j)) & 255)) for j in range(8))
    count = 2040 - sad                     # 8 * 255 - sum(255 - lo_X - hi_X)
    if trace is not None:
        trace.update(packed=word, lo_nibbles=_bytes_to_word(lo_n),
                     hi_nibbles=_bytes_to_word(hi_n), lo_lookup=lo_l, hi_lookup=hi_l,
                     lo_shifted=lo_s, hi_shifted=hi_s, lo_filled=lo_f, hi_masked=hi_m,
                     sad=sad, count=count)
    return count


def count_prefix(codes, x: int, t: int) -> int:
    """Occurrences of x among the first t symbols of a run of 2-bit codes, by the masking
    rule of Sec. 3: symbols at and past t are zeroed (they read as A) and, for x = A, the
    extra zeros are subtracted afterwards."""
    total = 0
    nwords = (len(codes) + 31) // 32
    for w in range(nwords):
        chunk = list(codes[32 * w:32 * w + 32])
        chunk += [0] * (32 - len(chunk))
        keep = max(0, min(32, t - 32 * w))
        masked = [c if j < keep else 0 for j, c in enumerate(chunk)]
        total += count_in_word(pack(masked), x)
    if x == 0:
        total -= 32 * nwords - t
    return total
