"""A plain executor of the tape format's arithmetic (test infrastructure):
leaf families are filled from given functions, bundles of FMAs, constants,
root accumulation and flushes run as the format defines them.  It checks the
compiler's scheduling, slot allocation and serialisation on the CPU; the
leaf arithmetic itself is the kernels' (checked on the GPU against the
oracle)."""
import collections
import struct

OP_GLEAF, OP_VLEAF, OP_RACC, OP_RFLUSH, OP_CONST, OP_NOP, OP_BUNDLE, OP_END = 2, 3, 4, 5, 6, 7, 8, 63


def decode_mask(mask, n_var):
    """The signed 2-bit coefficients of a leaf's momentum (0, +1, -1)."""
    out = []
    for j in range(n_var):
        c = (mask >> (2 * j)) & 3
        out.append({0: 0, 1: 1, 3: -1}[c])
    return tuple(out)


def run(data, g_leaf, v_leaf, gd_leaf=None, vd_leaf=None):
    """Execute a serialised tape.  g_leaf(mom, line_dst, line_src, j) and
    v_leaf(mom, j) give the j-th Taylor coefficient of a leaf (mom with the
    tape's sign), gd_leaf / vd_leaf its derivative in k_ext for families
    with the d/dk flag.  Returns {root index: {out line: accumulated value}}
    (the out line's phase left out)."""
    hdr = struct.unpack("<16I", data[:64])
    order, n_slots, n_instr, ins_off = hdr[2], hdr[5], hdr[6], hdr[8]
    words = struct.unpack("<%dQ" % n_instr, data[ins_off:ins_off + 8 * n_instr])
    S = [0.0] * n_slots
    S[1] = 1.0
    current = collections.defaultdict(float)
    roots = {}
    k = 0
    while k < n_instr:
        w = words[k]
        op = w & 63
        if op == OP_BUNDLE:
            n = (w >> 6) & 15
            res = []
            for q in words[k + 1:k + 1 + n]:
                d, a, b, c = q & 0xFFFF, (q >> 16) & 0xFFFF, (q >> 32) & 0xFFFF, q >> 48
                res.append((d, S[a] * S[b] + S[c]))
            for d, v in res:
                S[d] = v
            k += n + 1
            continue
        if op in (OP_GLEAF, OP_VLEAF):
            d, mask = (w >> 6) & 0x3FFF, (w >> 20) & 0x3FFF
            la, lb, M, dk = (w >> 34) & 7, (w >> 37) & 7, (w >> 40) & 7, (w >> 43) & 1
            mom = decode_mask(mask, order + 1)
            for j in range(M + 1):
                S[d + j] = g_leaf(mom, la, lb, j) if op == OP_GLEAF else v_leaf(mom, j)
                if dk:
                    S[d + M + 1 + j] = gd_leaf(mom, la, lb, j) if op == OP_GLEAF else vd_leaf(mom, j)
        elif op == OP_RACC:
            a, line = (w >> 20) & 0x3FFF, (w >> 34) & 7
            current[line] += S[a]
        elif op == OP_RFLUSH:
            roots[(w >> 6) & 0x3FFF] = dict(current)
            current.clear()
        elif op == OP_CONST:
            d = (w >> 6) & 0x3FFF
            S[d] = struct.unpack("<f", struct.pack("<I", w >> 32))[0]
        elif op == OP_END:
            break
        k += 1
    return roots
