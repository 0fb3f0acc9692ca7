"""Exact composition of discrete-library circuits, for pinning the FP64 oracle.

Every matrix entry of a CNOT/CV/CV^dag/H/T/T^dag circuit lies in Q(sqrt 2)(i).
Numbers here are kept exactly as (p + q*sqrt2) + i*(r + s*sqrt2) with
rational p, q, r, s.  Gates are applied to each column by the bit rule
(partner index = index with the target bit flipped, active when the control
bit is 1), not by Kronecker products, so this is an independent construction
of the same unitary.  Wire w is bit (n-1-w) of the basis index.
"""
from decimal import Decimal, getcontext
from fractions import Fraction

getcontext().prec = 60
_SQRT2 = Decimal(2).sqrt()


class QS2:
    """p + q*sqrt(2) with rational p, q."""
    __slots__ = ("p", "q")

    def __init__(self, p=0, q=0):
        self.p = Fraction(p)
        self.q = Fraction(q)

    def __add__(self, o):
        return QS2(self.p + o.p, self.q + o.q)

    def __sub__(self, o):
        return QS2(self.p - o.p, self.q - o.q)

    def __neg__(self):
        return QS2(-self.p, -self.q)

    def __mul__(self, o):
        return QS2(self.p * o.p + 2 * self.q * o.q, self.p * o.q + self.q * o.p)

    def is_zero(self):
        return self.p == 0 and self.q == 0

    def to_decimal(self):
        return Decimal(self.p.numerator) / Decimal(self.p.denominator) + \
            Decimal(self.q.numerator) / Decimal(self.q.denominator) * _SQRT2

    def exact_float(self):
        """float value when q == 0 and p is exactly representable, else None."""
        if self.q != 0:
            return None
        f = float(self.p)
        return f if Fraction(f) == self.p else None


class CX:
    """Complex number with QS2 real and imaginary parts."""
    __slots__ = ("re", "im")

    def __init__(self, re=None, im=None):
        self.re = re if re is not None else QS2()
        self.im = im if im is not None else QS2()

    def __add__(self, o):
        return CX(self.re + o.re, self.im + o.im)

    def __sub__(self, o):
        return CX(self.re - o.re, self.im - o.im)

    def __mul__(self, o):
        return CX(self.re * o.re - self.im * o.im, self.re * o.im + self.im * o.re)

    def to_complex(self):
        return complex(float(self.re.to_decimal()), float(self.im.to_decimal()))


ZERO = CX()
ONE = CX(QS2(1))
HALF = Fraction(1, 2)
# 1/sqrt(2) = sqrt(2)/2
INV_SQRT2 = QS2(0, HALF)


def u2(kind):
    """2x2 operator on the target wire: X, V, V^dag, H, T, T^dag."""
    if kind == "CNOT":
        return [[ZERO, ONE], [ONE, ZERO]]
    if kind in ("CV", "CVDG"):
        s = 1 if kind == "CV" else -1
        a = CX(QS2(HALF), QS2(s * HALF))   # (1 + s i)/2
        b = CX(QS2(HALF), QS2(-s * HALF))  # (1 - s i)/2
        return [[a, b], [b, a]]
    if kind == "H":
        h = CX(INV_SQRT2)
        return [[h, h], [h, CX(-INV_SQRT2)]]
    if kind in ("T", "TDG"):
        s = 1 if kind == "T" else -1
        w = CX(INV_SQRT2, QS2(0, s * HALF))  # e^{+- i pi/4}
        return [[ONE, ZERO], [ZERO, w]]
    raise ValueError(kind)


def apply_gate(n, col, kind, ctrl, tgt):
    """col <- G col for one column vector (list of CX) by the bit rule."""
    if kind == "I":
        return col
    U = u2(kind)
    tb = 1 << (n - 1 - tgt)
    out = list(col)
    for x in range(1 << n):
        if ctrl >= 0 and not (x >> (n - 1 - ctrl)) & 1:
            continue
        if x & tb:
            continue
        y = x | tb
        a, b = col[x], col[y]
        out[x] = U[0][0] * a + U[0][1] * b
        out[y] = U[1][0] * a + U[1][1] * b
    return out


def compose(n, gates):
    """gates: list of (kind, ctrl, tgt) applied first to last; returns S[i][j]."""
    N = 1 << n
    cols = []
    for j in range(N):
        col = [ONE if i == j else ZERO for i in range(N)]
        for kind, c, t in gates:
            col = apply_gate(n, col, kind, c, t)
        cols.append(col)
    return [[cols[j][i] for j in range(N)] for i in range(N)]


def trace_fitness(n, S, perm):
    """Eq. (11) evaluated exactly up to the final square roots (Decimal, 60 digits)."""
    N = 1 << n
    tr = CX()
    for j in range(N):
        s = S[perm[j]][j]
        tr = tr + CX(s.re, -s.im)
    m2 = (tr.re * tr.re + tr.im * tr.im).to_decimal()
    m = m2.sqrt() if m2 > 0 else Decimal(0)
    d = (Decimal(N) - m) / Decimal(N)
    if d < 0:
        d = Decimal(0)
    return float(Decimal(1) - d.sqrt())
