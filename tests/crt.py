"""Big-integer helpers for the oracle pins (plain Python ints)."""
from math import prod


def crt(residues, moduli):
    """The unique X in [0, prod(moduli)) with X = r_i mod m_i."""
    M = prod(moduli)
    x = 0
    for r, m in zip(residues, moduli):
        Mi = M // m
        x += int(r) * Mi * pow(Mi, -1, m)
    return x % M


def crt_columns(rows, moduli):
    """CRT of every column of a [len(moduli)][N] residue array."""
    N = len(rows[0])
    return [crt([int(rows[i][n]) for i in range(len(moduli))], moduli) for n in range(N)]


def centered(x, M):
    x %= M
    return x - M if x > M // 2 else x


def negacyclic_mul(a, b):
    """Schoolbook product in Z[X]/(X^N+1) of integer coefficient lists."""
    N = len(a)
    out = [0] * N
    for i in range(N):
        ai = int(a[i])
        if ai == 0:
            continue
        for j in range(N):
            k = i + j
            if k < N:
                out[k] += ai * int(b[j])
            else:
                out[k - N] -= ai * int(b[j])
    return out


def automorph_int(a, g):
    """a(X) -> a(X^g) in Z[X]/(X^N+1) on integer coefficient lists."""
    N = len(a)
    out = [0] * N
    for i in range(N):
        e = (i * g) % (2 * N)
        if e < N:
            out[e] += int(a[i])
        else:
            out[e - N] -= int(a[i])
    return out
