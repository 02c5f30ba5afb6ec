"""Order-free reference of the cubic tensor-product prolongation, shared by
the oracle pin and the GPU test (test infrastructure, no library code).

Vertex-centred refinement by two: fine index f along an axis sits at coarse
coordinate f / 2.  An even f is the coarse point f / 2 itself; an odd f is
the midpoint of coarse nodes c and c + 1 (c = (f - 1) // 2), where the cubic
Lagrange interpolant through nodes c - 1, c, c + 1, c + 2 has the weights
(-1, 9, 9, -1) / 16.  The value at a fine point is the sum, over the tensor
product of the three axes' nodes, of the weight products times the coarse
data (periodic coarse indices), rounded ONCE (math.fsum): an evaluation
that shares no order or structure with any nested one."""
import math


def cubic_nodes(f: int):
    """(coarse indices, weights) of fine index f along one axis."""
    if f % 2 == 0:
        return [f // 2], [1.0]
    c = (f - 1) // 2
    return [c - 1, c, c + 1, c + 2], [-1 / 16, 9 / 16, 9 / 16, -1 / 16]


def tensor_sum_exact(data, p) -> float:
    """Prolongated value at fine point p = (x, y, z) from coarse data of
    shape (nz, ny, nx), every product exact in the sum's terms and the sum
    rounded once."""
    nz, ny, nx = data.shape
    (ix, wx), (iy, wy), (iz, wz) = (cubic_nodes(int(p[d])) for d in range(3))
    terms = []
    for a in range(len(iz)):
        for b in range(len(iy)):
            for c in range(len(ix)):
                v = float(data[iz[a] % nz, iy[b] % ny, ix[c] % nx])
                # each weight is k / 16 with k in {-1, 9, 16}, so the product of
                # the three is K / 4096 with |K| <= 4096 an exact integer; K * v
                # may round, so it enters fsum as two parts that are exact
                k = round(wz[a] * 16) * round(wy[b] * 16) * round(wx[c] * 16)
                terms.extend(_exact_product(k, v, 4096))
    return math.fsum(terms)


def _exact_product(k: int, v: float, scale: int):
    """k * v / scale as a list of floats whose exact sum is the exact value
    (|k| <= 4096, at most 13 bits; scale a power of two)."""
    if k == 0 or v == 0.0:
        return [0.0]
    # split v into a high part of 26 significant bits and the exact rest (at
    # most 27 bits): each part times k (<= 13 bits) is then exact in a double
    m, e = math.frexp(v)
    hi = math.ldexp(math.floor(math.ldexp(m, 26)), e - 26)
    lo = v - hi
    return [(k * hi) / scale, (k * lo) / scale]
