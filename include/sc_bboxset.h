/*
 * sc_bboxset.h -- host-side bounding-box-set algebra of libsc_level.so.
 *
 * A bboxset is a set of points of a uniform 3D grid, stored as its discrete
 * derivative (arXiv 1308.1343, Sec. 2.2, "Discrete Derivatives of Bounding
 * Box Sets"): along each axis, membership changes between p - e_d and p
 * are recorded, by dimensional recursion, in ordered maps of
 * lower-dimensional sets (Sec. 2.3, "Implementation").  Set operations are
 * evaluated by the sweep of Sec. 2.3 (Fig. "bboxset-traverse"): the sweep
 * line advances through the stored derivative positions of both operands,
 * keeping their current cross-sections, and stores the change of the
 * result's cross-section.  The symmetric difference is computed directly on
 * the stored derivatives (Eq. "xor").
 *
 * These entry points exist so that the algebra can be checked against
 * brute-force point enumeration; the level runtime uses the same C++ code
 * internally to validate levels and build ghost-exchange lists.
 *
 * Boxes are int64_t[6] = {lo.x, lo.y, lo.z, hi.x, hi.y, hi.z}, half-open.
 * Host memory only, thread-safe, no CUDA.  Return SC_OK or SC_EINVAL
 * (lo > hi, NULL pointer with nonzero count, unknown op); results larger
 * than cap are counted in *n but not written.
 */
#ifndef SC_BBOXSET_H
#define SC_BBOXSET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SC_SET_UNION 0        /* A | B */
#define SC_SET_INTERSECTION 1 /* A & B */
#define SC_SET_DIFFERENCE 2   /* A \ B */
#define SC_SET_XOR 3          /* A ^ B (symmetric difference) */

/* T = A op B; writes T's normalized box list: disjoint boxes, z-slabs of
 * constant cross-section from the outer sweep, then y-slabs, then x-runs,
 * vertically merged where a box continues unchanged; deterministic. */
int sc_bboxset_op(int32_t op, const int64_t* a, int64_t na, const int64_t* b,
                  int64_t nb, int64_t* out, int64_t cap, int64_t* n);

/* Points of the full derivative d_x d_y d_z of the union of the boxes
 * (stored form of the set), as int64_t[3] triples sorted by (z, y, x).  For
 * one box these are its 8 corners {lo, hi}^3. */
int sc_bboxset_derivative(const int64_t* a, int64_t na, int64_t* pts, int64_t cap,
                          int64_t* n);

/* Grow the union of the boxes by lo_by[d] / hi_by[d] points along each
 * axis (Sec. 2's `expand`) and shift it by v (Sec. 2's `shift`), in that
 * order; writes the normalized box list. */
int sc_bboxset_expand_shift(const int64_t* a, int64_t na, const int64_t lo_by[3],
                            const int64_t hi_by[3], const int64_t v[3], int64_t* out,
                            int64_t cap, int64_t* n);

/* Spacing change (Sec. 2): the points c of a grid with `ratio` times the
 * spacing, sharing the origin, that coincide with points of the union of
 * the boxes: {c : ratio * c in A} (vertex-centred).  Writes the normalized
 * box list.  Errors: SC_EINVAL for ratio < 1. */
int sc_bboxset_coarsen(const int64_t* a, int64_t na, int64_t ratio, int64_t* out, int64_t cap,
                       int64_t* n);

/* Number of points of the union of the boxes (the union, not the sum). */
int sc_bboxset_size(const int64_t* a, int64_t na, int64_t* npoints);

#ifdef __cplusplus
}
#endif
#endif /* SC_BBOXSET_H */
