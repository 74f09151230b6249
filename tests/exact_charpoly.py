"""Exact characteristic-polynomial roots for small symmetric matrices (test pin, pure Python).

Every float64 is a dyadic rational, so H = G J G^T built from Fractions of the float64 entries is
exact; its characteristic polynomial comes from the Faddeev-LeVerrier recursion in Fractions,
Yun's square-free factorization gives the multiplicities, and the real roots of each square-free
factor are isolated by Sturm sequences and bisected in exact arithmetic.
"""
from fractions import Fraction


def mat_mul(A, B):
    n, k, m = len(A), len(B), len(B[0])
    return [[sum(A[i][r] * B[r][j] for r in range(k)) for j in range(m)] for i in range(n)]


def charpoly(A):
    """Coefficients c[0..n] of det(x I - A) = sum c_k x^(n-k), c[0] = 1 (Faddeev-LeVerrier)."""
    n = len(A)
    c = [Fraction(1)]
    M = [[Fraction(0)] * n for _ in range(n)]
    for k in range(1, n + 1):
        # M_k = A M_{k-1} + c_{k-1} I ;  c_k = -tr(A M_k) / k
        M = mat_mul(A, M) if k > 1 else [[Fraction(0)] * n for _ in range(n)]
        for i in range(n):
            M[i][i] += c[k - 1]
        AM = mat_mul(A, M)
        c.append(-sum(AM[i][i] for i in range(n)) / k)
    return c


def _trim(p):
    while len(p) > 1 and p[0] == 0:
        p = p[1:]
    return p


def poly_divmod(a, b):
    a, b = _trim(list(a)), _trim(list(b))
    if len(a) < len(b):
        return [Fraction(0)], a
    q = [Fraction(0)] * (len(a) - len(b) + 1)
    r = list(a)
    for i in range(len(q)):
        coef = r[i] / b[0]
        q[i] = coef
        for j in range(len(b)):
            r[i + j] -= coef * b[j]
    rem = _trim(r[len(q):]) if len(r) > len(q) else [Fraction(0)]
    return q, rem


def poly_gcd(a, b):
    a, b = _trim(list(a)), _trim(list(b))
    while not (len(b) == 1 and b[0] == 0):
        _, r = poly_divmod(a, b)
        a, b = b, r
    return [x / a[0] for x in a]


def deriv(p):
    n = len(p) - 1
    return [p[i] * (n - i) for i in range(n)] or [Fraction(0)]


def evalp(p, x):
    v = Fraction(0)
    for c in p:
        v = v * x + c
    return v


def squarefree(p):
    """Yun: list of (multiplicity, square-free factor)."""
    out = []
    a = poly_gcd(p, deriv(p))
    b, _ = poly_divmod(p, a)
    c, _ = poly_divmod(deriv(p), a)
    d = [ci - di for ci, di in zip([Fraction(0)] * (max(len(c), len(deriv(b))) - len(c)) + c,
                                   [Fraction(0)] * (max(len(c), len(deriv(b))) - len(deriv(b))) + deriv(b))]
    i = 1
    while len(_trim(b)) > 1:
        aa = poly_gcd(b, d)
        if len(_trim(aa)) > 1:
            out.append((i, aa))
        b, _ = poly_divmod(b, aa)
        c, _ = poly_divmod(d, aa)
        db = deriv(b)
        L = max(len(c), len(db))
        d = [x - y for x, y in zip([Fraction(0)] * (L - len(c)) + c, [Fraction(0)] * (L - len(db)) + db)]
        i += 1
    return out


def sturm_chain(p):
    chain = [_trim(p), _trim(deriv(p))]
    while len(chain[-1]) > 1 or chain[-1][0] != 0:
        _, r = poly_divmod(chain[-2], chain[-1])
        if len(r) == 1 and r[0] == 0:
            break
        chain.append([-x for x in r])
    return chain


def sign_changes(chain, x):
    vals = [evalp(p, x) for p in chain]
    vals = [v for v in vals if v != 0]
    return sum(1 for a, b in zip(vals, vals[1:]) if (a < 0) != (b < 0))


def real_roots(p, bits=120):
    """Real roots of a square-free polynomial, as Fractions accurate to 2^-bits relative-ish."""
    chain = sturm_chain(p)
    bound = 1 + max(abs(c / p[0]) for c in p[1:]) if len(p) > 1 else Fraction(1)
    lo, hi = -bound, bound
    roots = []

    def count(a, b):
        return sign_changes(chain, a) - sign_changes(chain, b)

    stack = [(lo, hi)]
    while stack:
        a, b = stack.pop()
        c = count(a, b)
        if c == 0:
            continue
        if c == 1:
            for _ in range(bits):
                mid = (a + b) / 2
                if count(a, mid) == 1:
                    b = mid
                else:
                    a = mid
            roots.append((a + b) / 2)
            continue
        mid = (a + b) / 2
        stack.append((a, mid))
        stack.append((mid, b))
    return sorted(roots)


def eigenvalues_exact(H):
    """Sorted eigenvalues (with multiplicity) of a symmetric matrix of Fractions."""
    p = charpoly(H)
    out = []
    for mult, f in squarefree(p):
        for r in real_roots(f):
            out += [r] * mult
    return sorted(out)
