// Plain descriptor structs shared by the host runtime and the kernels.
#pragma once

namespace sc {
namespace dev {

// ---------------------------------------------------------------------------
// Descriptors (built on the host, uploaded once per level)
// ---------------------------------------------------------------------------

struct DBox {
  long long off;  // element index of the interior corner (0,0,0)
  long long py;   // row pitch (elements)
  long long pz;   // plane pitch (elements)
  int nx, ny, nz; // interior extent
  int dom;        // domain index
  int wrap;       // bit 0: the box alone tiles a domain periodic on every
                  // axis (nx even, nx and ny >= 2), so the stencil kernels read
                  // the periodic images of its interior in x and y directly;
                  // bit 1: also nz >= 2, and the warp-specialised kernels read
                  // its z ghosts the same way (the one-role kernels have them
                  // gathered)
};

struct DItem {
  int box;
  int x0, y0, z0;  // tile origin (interior coordinates of the box)
  int nzr;         // number of planes of the z-run
  int txh;         // threads per tile row; tile is (2*txh) x (NT/txh) points
};

// A rectangle of points of one field, for gathers and reductions.
struct DRect {
  long long src, dst;        // element index of the first point (dst unused
                             // by reductions)
  long long spy, spz;        // source pitches
  long long dpy, dpz;        // destination pitches
  int ex, ey, ez;            // extent
  int dom;                   // domain of the points
  int box;                   // box of the points (interior rectangles)
  int x0, y0, z0;            // interior coordinates of the first point
  int pairs;                 // gathers: 1 if ex, src and dst are even, so the
                             // rectangle is copied in 16-byte pairs of x-points
                             // (its chunks then count pairs, not points)
};

// A set of fine points that prolongation fills (interior points of one fine
// box, or ghost points of its shell), all of one index parity per axis (so
// spaced 2 apart along every axis) and all drawing on the interior of one
// coarse box.
struct DProl {
  long long dst;       // fine element index of the first point
  int dpy, dpz;        // fine box pitches
  int ex, ey, ez;      // number of points per axis (stride 2)
  int fx0, fy0, fz0;   // fine level index of the first point
  long long cbase;     // coarse element index of coarse level index (0, 0, 0)
                       // in the coarse box's layout (may lie outside the box)
  int cpy, cpz;        // coarse box pitches
};

// Prolongation runs one CTA per tile of kProlTX x kProlTY x kProlTZ points of
// a DProl entry; its chunk list holds (entry, tile index) pairs.
constexpr int kProlTX = 16, kProlTY = 8, kProlTZ = 4;

// A rectangle of coarse points that restriction sets from fine points 2c.
struct DRestr {
  long long dst;       // coarse element index of the first point
  int dpy, dpz;        // coarse box pitches
  int ex, ey, ez;      // extent
  long long src;       // fine element index of the fine point under the first
  int spy, spz;        // fine box pitches (the source advances by 2 per point)
};

// One ghost copy seen from its source: the source rectangle in the source
// box's interior coordinates [lo, hi) and where its first point goes.  A
// producer that writes point (x, y, z) of the source box inside the
// rectangle also writes it to dbase + (x-lo0) + (y-lo1)*dpy + (z-lo2)*dpz.
struct DPush {
  int lo0, lo1, lo2, hi0, hi1, hi2;
  int dbase, dpy, dpz;
  int pad[3];
};

// One ghost copy into an x face of a box, read by the warp-specialised
// kernels from its owner directly instead of being gathered (the copy's rows
// are two points, 16 bytes, wide: half of every DRAM sector at both ends of
// a gather).  In the destination box's interior coordinates it fills the
// ghost pair of rows y in [y0, y1) of planes z in [z0, z1); the source of
// row y0 of plane z0 is element src, and the source pitches are spy, spz.
// sbox names the source box (bounds checks of the checked build).
struct DXGhost {
  int y0, y1, z0, z1;
  int src, spy, spz, sbox;
};

// One ghost copy that crosses ranks of a distributed level, seen from this
// rank: a rectangle of the local field (interior points of a local source
// box when packing, ghost points of a local destination box when unpacking)
// and its place in the contiguous exchange buffer, where the rectangle's
// points follow each other x fastest.  The buffer holds two fields: the
// second one's copy of a point sits `second` doubles after the first's.
struct DXfer {
  long long fld;   // element index of the first point in the field
  long long buf;   // index of the first point in the exchange buffer
  long long fpy, fpz;  // field pitches of the rectangle's box
  int ex, ey, ez;  // extent
  int dom;         // domain of the points
  int second;      // offset of the second field's block (the peer's points)
  int pad;
};

// A chunk of up to CHUNK consecutive points of one rectangle.
struct DChunk {
  int rect;
  int first;  // index of the first point within the rectangle (x fastest)
};

constexpr int kChunk = 1024;  // reductions and pointwise kernels
constexpr int kGatherChunk = 256;  // ghost gather: one point per thread

// Error bits of the device error word.
constexpr unsigned kErrNonFinite = 1u;   // Inf/NaN reached the fixed-point path
constexpr unsigned kErrScale = 2u;       // an input exceeded its domain bound
constexpr unsigned kErrBounds = 4u;      // checked build: an index left its box
constexpr unsigned kErrTimeout = 8u;     // a bounded wait inside a kernel gave up

}  // namespace dev
}  // namespace sc
