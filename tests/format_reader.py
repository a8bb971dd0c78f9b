"""A second, deliberately naive reader of the stream format, for cross-checks.

Written from the format definition alone (Sec. 2.1 of Cloud et al. and the
readings R3-R6 and R14 stated in the oracle), in pure Python, sharing no code
with the oracle or the CUDA library.  It is only meant for small streams.
"""
import struct


def read_container(stream: bytes) -> dict:
    if stream[:4] != b"HZB1":
        raise ValueError("bad magic")
    flags, n, B, nb = struct.unpack_from("<IQII", stream, 4)
    lengths = list(stream[24:280])
    pos = 280
    index = None
    if flags & 1:
        index = list(struct.unpack_from(f"<{nb}I", stream, pos))
        pos += 4 * nb
    sub, S = None, 0
    if flags & 2:
        if not flags & 1 or flags & ~3:
            raise ValueError("sub-block offsets come only with the index")
        # S, then for each block the bit offsets of its symbols S, 2S, ..., (B/S - 1)S
        S = struct.unpack_from("<I", stream, pos)[0]
        if S < 32 or S % 32 or B % S:
            raise ValueError("bad sub-block size")
        per = B // S - 1
        flat = struct.unpack_from(f"<{nb * per}I", stream, pos + 4)
        sub = [list(flat[k * per:(k + 1) * per]) for k in range(nb)]
        pos += 4 + 4 * nb * per
    records = []
    off = 0
    for _ in range(nb):
        bits = struct.unpack_from("<I", stream, pos + 4 * off)[0]
        nwords = (bits + 31) // 32
        words = list(struct.unpack_from(f"<{nwords}I", stream, pos + 4 * off + 4))
        records.append({"word_offset": off, "bits": bits, "words": words})
        off += 1 + nwords
    return {"flags": flags, "n": n, "B": B, "nb": nb, "lengths": lengths, "index": index,
            "S": S, "sub": sub, "records": records, "end": pos + 4 * off}


def code_table(lengths) -> dict:
    """{(length, value): symbol} for canonical codes (RFC 1951 3.2.2 order)."""
    table = {}
    code, prev = -1, 0
    for sym_len, sym in sorted((l, s) for s, l in enumerate(lengths) if l > 0):
        code = 0 if code < 0 else (code + 1) << (sym_len - prev)
        prev = sym_len
        table[(sym_len, code)] = sym
    return table


def decode(stream: bytes) -> bytes:
    c = read_container(stream)
    table = code_table(c["lengths"])
    out = bytearray()
    for k, rec in enumerate(c["records"]):
        want = min(c["B"], c["n"] - k * c["B"])
        bitstr = "".join(f"{w:032b}" for w in rec["words"])
        p, got = 0, 0
        starts = []  # bit position of every symbol's code
        while got < want:
            starts.append(p)
            v, l = 0, 0
            while (l, v) not in table:
                v = (v << 1) | int(bitstr[p])
                l += 1
                p += 1
                if l > 64 or p > rec["bits"]:
                    raise ValueError("bad code")
                if (l, v) in table:
                    break
            out.append(table[(l, v)])
            got += 1
        if p != rec["bits"] or "1" in bitstr[p:]:
            raise ValueError("bad block end")
        if c["sub"] is not None:
            for j, e in enumerate(c["sub"][k], start=1):
                at = j * c["S"]
                if e != (starts[at] if at < want else rec["bits"]):
                    raise ValueError("bad sub-block offset")
    return bytes(out)
