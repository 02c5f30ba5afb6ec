/*
 * sc_dist.h -- a level distributed over ranks (one GPU each): C ABI of
 * libsc_level.so, beside sc_level.h.
 *
 * The paper's infrastructure distributes the boxes of a refinement level
 * over processes and derives the communication schedule -- which points
 * every process sends to and receives from every other -- from bboxset
 * intersections (arXiv 1308.1343, Sec. 2, "Efficient Bounding Box Algebra":
 * the list of operations built on the set algebra, and the motivation of
 * bboxsets by the distribution of a level over many processes).  Here:
 *
 *  - sc_dist_partition assigns whole boxes to ranks, balanced by point
 *    count;
 *  - sc_dist_create builds one rank's part of the level: a level object
 *    (usable with the sc_level_* queries, layout and configuration calls)
 *    that stores only this rank's boxes, keeps the ghost copies between
 *    them as its local exchange list, and splits the copies that cross
 *    ranks into per-peer send and receive lists;
 *  - per RK4 step (two RK4 stages per stencil pass, see
 *    sc_level_set_fusion), the ghosts of the two stencil inputs of each
 *    pass cross ranks once: sc_dist_pack writes the face slabs other ranks
 *    read into a contiguous send buffer, the caller moves each peer's part
 *    to that peer (NCCL grouped send/recv, or any transport), and
 *    sc_dist_unpack writes what arrived into this rank's own ghost points;
 *  - the loss of sc_level_misfit is this rank's share; the caller sums it
 *    over ranks (one scalar all-reduce).  g_c2 and g_u0 would stay local;
 *    the adjoint is not distributed here (sc_level_grad refuses a
 *    distributed level).
 *
 * Exchange buffers (caller-owned DEVICE memory, doubles): one block per
 * peer, in increasing peer rank, at the offset sc_dist_peer reports.  A
 * peer's block holds 2 * points doubles: first the first field's values,
 * then the second field's, each as the peer's ghost copies in list order
 * (sc_dist_list), the points of one copy x fastest, then y, then z.  The
 * sender's send block for a peer and the receiver's receive block for the
 * sender have the same length and layout, so the transport copies bytes.
 *
 * Arithmetic: the same kernels as sc_level_rk4_step.  In the fixed-point
 * form each rank's exponent bound of a field is the largest over its own
 * boxes and the ghost values it received (sc_dist_unpack raises it), so
 * results can differ from a one-GPU run in the last bits but stay within
 * the form's bound; in SC_ARITH_FP64 they are bit-identical to it.
 * Restrictions: every domain periodic on every axis, two stages per pass
 * (fixed at creation), batched launches (no CUDA graph: the transport runs
 * between the passes).
 */
#ifndef SC_DIST_H
#define SC_DIST_H

#include <stdint.h>

#include "sc_level.h"

#ifdef __cplusplus
extern "C" {
#endif

#define SC_DIST_GREEDY 0 /* balance only: largest boxes first, each to the
                            least-loaded rank                             */
#define SC_DIST_BISECT 1 /* recursive bisection in space by point count:
                            neighbouring boxes share a rank               */

/* Assign each of nboxes boxes a rank in [0, nranks): rank_of_box[b] (host
 * array of nboxes).  Every rank gets at least one box.  Deterministic.
 * Errors: SC_EINVAL (nranks < 1, nranks > nboxes, NULL pointers, unknown
 * method). */
int sc_dist_partition(const sc_box* boxes, int32_t nboxes, int32_t nranks, int32_t method,
                      int32_t* rank_of_box);

/* Rank `rank`'s part of the level (boxes, doms, ghost as sc_level_create,
 * validated as a whole).  rank_of_box: the partition (host, nboxes
 * entries), e.g. from sc_dist_partition; every rank must own a box.  The
 * new level stores this rank's boxes in increasing whole-level index
 * (sc_dist_global_box maps them back); its field buffers, layout and
 * exchange list cover those boxes only.  Free with sc_level_destroy.
 * Errors: SC_EINVAL, SC_ENOMEM. */
int sc_dist_create(const sc_box* boxes, int32_t nboxes, const sc_domain* doms, int32_t ndoms,
                   int32_t ghost, const int32_t* rank_of_box, int32_t nranks, int32_t rank,
                   sc_level** out);

/* rank, number of ranks and number of peers (ranks this one exchanges
 * ghost points with) of a distributed level; a level from sc_level_create
 * reports rank 0 of 1 with no peers. */
int sc_dist_info(const sc_level* level, int32_t* rank, int32_t* nranks, int32_t* npeers);

/* Whole-level index of local box `box`. */
int sc_dist_global_box(const sc_level* level, int32_t box, int32_t* global_box);

/* Sizes in doubles of the send and receive buffers (both fields). */
int sc_dist_buffer_sizes(const sc_level* level, int64_t* send_doubles, int64_t* recv_doubles);

/* Peer i (0 <= i < npeers, increasing rank): its rank, the points of one
 * field this rank sends to / receives from it, and the offsets (doubles) of
 * its blocks in the send / receive buffers. */
int sc_dist_peer(const sc_level* level, int32_t i, int32_t* peer, int64_t* send_points,
                 int64_t* recv_points, int64_t* send_offset, int64_t* recv_offset);

/* Host copy of peer i's ghost copies (recv == 0: those this rank sends,
 * src_box local and dst_box the peer's box as a whole-level index;
 * recv != 0: those it receives, dst_box local and src_box whole-level),
 * coordinates in the level's index space as in sc_level_exchange_list;
 * *n receives the count (cap = 0 to size). */
int sc_dist_list(const sc_level* level, int32_t i, int32_t recv, sc_copy* out, int64_t cap,
                 int64_t* n);

/* Which pair of fields an exchange moves. */
#define SC_DIST_STATE 0 /* the state (u, pi) passed in: before pass A      */
#define SC_DIST_STAGE 1 /* the library's stage fields w_2 (u and pi are
                           ignored, pass NULL): between pass A and pass B */

/* Pack the send buffer (sc_dist_buffer_sizes doubles, device) from the
 * interior points of this rank's boxes.  One launch on `stream`. */
int sc_dist_pack(sc_level* level, int32_t which, const double* u, const double* pi,
                 double* send, void* stream);

/* Write the receive buffer into the ghost points of this rank's boxes that
 * other ranks own, and raise the fixed-point exponent bounds the next pass
 * reads to cover them.  One launch on `stream`.  A non-finite value is
 * reported by the next pass (SC_EDEVICE at sc_level_sync). */
int sc_dist_unpack(sc_level* level, int32_t which, const double* recv, double* u, double* pi,
                   void* stream);

/* Start a run of RK4 steps on (u, pi) with wave speed c2 and step dt (ndt
 * entries: 1 or one per domain), as sc_level_rk4_step would: the pre-scaled
 * wave speeds and the exponent bounds of this rank's interior.  Then, per
 * step:
 *   sc_dist_pack(SC_DIST_STATE) -> transport -> sc_dist_unpack(SC_DIST_STATE)
 *   sc_dist_rk4_pass(0)   (local ghost gather of (u, pi), then pass A)
 *   sc_dist_pack(SC_DIST_STAGE) -> transport -> sc_dist_unpack(SC_DIST_STAGE)
 *   sc_dist_rk4_pass(1)   (local ghost gather of w_2, then pass B: u, pi
 *                          hold the step's result)
 * Out-of-order passes return SC_EINVAL.  u, pi, c2 must stay the same
 * buffers for the whole run. */
int sc_dist_rk4_begin(sc_level* level, double* u, double* pi, const double* c2,
                      const double* dt, int32_t ndt, void* stream);
int sc_dist_rk4_pass(sc_level* level, double* u, double* pi, int32_t pass, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SC_DIST_H */
