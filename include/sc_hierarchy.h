/* Two-level refinement hierarchy over the level library: prolongation,
 * restriction and Berger-Oliger time stepping (arXiv 1308.1343, Sec. 2:
 * the AMR operators a refinement level derives from the bboxset algebra).
 *
 * The paper names these operators but does not define them; the library's
 * readings are:
 *  - Vertex-centred refinement by 2, both levels sharing the index origin:
 *    fine index f (per axis) lies at coarse coordinate f / 2.
 *  - Prolongation: cubic Lagrange interpolation along each axis as a tensor
 *    product (weights (-1, 9, 9, -1) / 16 at odd fine indices, injection at
 *    even ones; exact for polynomials of degree <= 3 per axis), evaluated as
 *    successive one-dimensional interpolations along z, then y, then x, of
 *    data interpolated linearly in time between two coarse time levels.
 *  - Restriction: injection, coarse point c takes the fine value at 2c.
 *  - Time stepping (sub-cycling): one hierarchy step of dt is one coarse
 *    RK4 step of dt, two fine RK4 steps of dt/2 (before each, the fine
 *    buffer band and ghost shell are prolongated from the coarse levels at t
 *    and t + dt, at alpha = 0 and 1/2), and restriction of the fine trusted
 *    region T into the coarse level.
 *
 * Levels: the coarse level has one domain, periodic on every axis; the fine
 * level has one domain R (fine index space, spacing h/2), periodic on no
 * axis, tiled by its boxes.  The buffer band is the outer `buffer` (>= 4)
 * points of R; T is R shrunk by `buffer`.  One RK4 step changes a point from
 * data within 4 points, so T only depends on data the scheme maintains; the
 * band's values after a fine step are boundary-influenced and are replaced
 * by the next prolongation.
 *
 * Fields: caller-owned DEVICE buffers in each level's layout
 * (sc_level_field_size doubles, see sc_level.h).  The hierarchy does not own
 * the levels; destroy it before them.  Errors: SC_EINVAL (message says
 * which rule failed), SC_ENOMEM, SC_ECUDA. */
#ifndef SC_HIERARCHY_H
#define SC_HIERARCHY_H

#include <stdint.h>

#include "sc_level.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sc_hierarchy sc_hierarchy;

/* Build the prolongation and restriction lists with the bboxset algebra:
 * targets = (R union its star-shaped ghost shell) minus T, per fine box
 * (interior points and the shell points outside R), split so that every
 * point's 4x4x4 (or smaller) coarse stencil lies inside ONE coarse box's
 * interior; restriction = the coarse points c with 2c in T (bboxset
 * spacing change), per (coarse box, fine box) pair.
 * Errors (SC_EINVAL): refinement ratio other than 2; buffer < 4; a level
 * with more than one domain; a coarse domain not periodic on every axis or
 * a fine domain periodic on any; fine spacing not half the coarse; T empty;
 * a target whose stencil lies in no coarse box interior. */
int sc_hierarchy_create(sc_level* coarse, sc_level* fine, int32_t ratio, int32_t buffer,
                        sc_hierarchy** out);
void sc_hierarchy_destroy(sc_hierarchy* hierarchy);

/* Number of fine points prolongation fills and of coarse points
 * restriction sets. */
int sc_hierarchy_counts(const sc_hierarchy* hierarchy, int64_t* n_prolong,
                        int64_t* n_restrict);

/* The points themselves, host int64_t (x, y, z) triples in each level's
 * index space (at most cap; *n = total).  For tests. */
int sc_hierarchy_prolongation_points(const sc_hierarchy* hierarchy, int64_t* xyz, int64_t cap,
                                     int64_t* n);
int sc_hierarchy_restriction_points(const sc_hierarchy* hierarchy, int64_t* xyz, int64_t cap,
                                    int64_t* n);

/* Fill the fine targets of fu and fpi by prolongation from the coarse
 * levels (u0, p0) at time t and (u1, p1) at t + dt, at time t + alpha dt.
 * Coarse ghosts are not read.  Enqueued on the stream. */
int sc_hierarchy_prolongate(sc_hierarchy* hierarchy, const double* u0, const double* u1,
                            const double* p0, const double* p1, double alpha, double* fu,
                            double* fpi, void* stream);

/* Coarse points c with 2c in T take the fine values (both fields).
 * Enqueued on the stream. */
int sc_hierarchy_restrict(sc_hierarchy* hierarchy, const double* fu, const double* fpi,
                          double* cu, double* cpi, void* stream);

/* nsteps hierarchy steps of dt (see the top of this header) on the coarse
 * fields (cu, cpi, cc2) and the fine fields (fu, fpi, fc2), in place.  mode
 * is the levels' launch mode (SC_MODE_*).  c2 ghosts need not be filled.
 * Library-owned scratch: four coarse fields (the coarse level at t and its
 * time interpolation, written only where prolongation reads them). */
int sc_hierarchy_step(sc_hierarchy* hierarchy, double* cu, double* cpi, const double* cc2,
                      double* fu, double* fpi, const double* fc2, double dt, int32_t nsteps,
                      int32_t mode, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SC_HIERARCHY_H */
