// Index arithmetic of the tiled kernels: the D2Q9 directions, which node a
// thread updates, where its streaming sources and finite-difference taps lie,
// which shared-memory and boundary side-array entries it touches, how the
// frame tiles are enumerated and where the TMA boxes start.  Plain C++ with
// no device code: the kernels call these functions, and a host program
// (tests/c/tile_bounds.cc) drives them over every tile shape and over ragged
// and degenerate lattices to check each index against its allocation.
//
// The lattice type G of the templates is anything with the members
//   nx, ny (nodes), pitch (row pitch in elements), per_x, per_y (periodic
//   axes) and blen (entries per edge of the side array),
// e.g. the kernels' Params.
#pragma once
#include <stddef.h>

#ifdef __CUDACC__
#define LBS_HD __host__ __device__ __forceinline__
#else
#define LBS_HD inline
#endif

namespace lbs {

enum { kLeft = 0, kRight = 1, kBottom = 2, kTop = 3 };

// ------------------------------------------------------------------ D2Q9
// Tab. 1: c_q = c (ex(q), ey(q)); q = 0 rest, 1-4 axes (+x, +y, -x, -y),
// 5-8 diagonals (+x+y, -x+y, -x-y, +x-y); opp(q) is the reversed direction
LBS_HD constexpr int ex(int q) { return (q == 1 || q == 5 || q == 8) ? 1 : ((q == 3 || q == 6 || q == 7) ? -1 : 0); }
LBS_HD constexpr int ey(int q) { return (q == 2 || q == 5 || q == 6) ? 1 : ((q == 4 || q == 7 || q == 8) ? -1 : 0); }
LBS_HD constexpr int opp(int q) { return q == 0 ? 0 : (q <= 4 ? ((q + 1) % 4) + 1 : ((q - 3) % 4) + 5); }

// ------------------------------------------------------------------ tiles
// A thread block owns a TX x TY tile of nodes with NTY thread rows; each
// thread handles CPT = TY / NTY nodes of one column (thread t: column t % TX,
// rows t / TX + i NTY).  Shared memory holds u on the tile plus a 2-node halo
// (R2, R2W x R2H) and N on the tile plus a 1-node halo (R1, R1W x R1H); NRING
// is the number of R2 entries outside the tile.
template <int TX_, int TY_, int NTY_>
struct TileGeom {
  static constexpr int TX = TX_, TY = TY_, NTY = NTY_;
  static constexpr int NT = TX * NTY, CPT = TY / NTY;
  static constexpr int R2W = TX + 4, R2H = TY + 4, R1W = TX + 2, R1H = TY + 2;
  static constexpr int NRING = R2W * R2H - TX * TY;
  static_assert(TY % NTY == 0, "tile rows must split evenly over thread rows");
};

// position (rx, ry) in R2 of ring entry r in [0, NRING): two full rows below
// the tile, two full rows above it, then two columns on each side
template <class C>
LBS_HD void ring_pos(int r, int &rx, int &ry) {
  constexpr int top = 2 * C::R2W;
  if (r < top) {
    ry = r / C::R2W;
    rx = r % C::R2W;
  } else if (r < 2 * top) {
    r -= top;
    ry = C::TY + 2 + r / C::R2W;
    rx = r % C::R2W;
  } else {
    r -= 2 * top;
    ry = 2 + r / 4;
    const int c = r % 4;
    rx = c < 2 ? c : C::TX + c;
  }
}

// wrap (periodic axis) or reject a node coordinate; false outside a wall.
// Coordinates handed in lie within one lattice length of the lattice.
template <class G>
LBS_HD bool locate(const G &P, int &x, int &y) {
  if (x < 0 || x >= P.nx) {
    if (!P.per_x) return false;
    x = (x + P.nx) % P.nx;
  }
  if (y < 0 || y >= P.ny) {
    if (!P.per_y) return false;
    y = (y + P.ny) % P.ny;
  }
  return true;
}

// Source (sx, sy) of population q streaming into node (x, y) of the lattice:
// (x - ex(q), y - ey(q)), wrapped on a periodic axis.  False where the source
// lies beyond a wall (the boundary rules then supply f_q).
template <class G>
LBS_HD bool stream_source(const G &P, int x, int y, int q, int &sx, int &sy) {
  sx = x - ex(q);
  sy = y - ey(q);
  bool in = true;
  if (sx < 0 || sx >= P.nx) {
    if (P.per_x) sx = sx < 0 ? sx + P.nx : sx - P.nx;
    else in = false;
  }
  if (sy < 0 || sy >= P.ny) {
    if (P.per_y) sy = sy < 0 ? sy + P.ny : sy - P.ny;
    else in = false;
  }
  return in;
}

// Whether the outgoing link opp(q) of node (x, y) crosses the x wall (ox) or
// the y wall (oy): exactly the directions q whose source stream_source finds
// beyond a wall.
template <class G>
LBS_HD void link_crosses(const G &P, int x, int y, int q, bool &ox, bool &oy) {
  ox = !P.per_x && ((ex(q) == 1 && x == 0) || (ex(q) == -1 && x == P.nx - 1));
  oy = !P.per_y && ((ey(q) == 1 && y == 0) || (ey(q) == -1 && y == P.ny - 1));
}

// walls node (x, y) lies on: xw = kLeft / kRight or -1, yw = kBottom / kTop or -1
template <class G>
LBS_HD void walls_of(const G &P, int x, int y, int &xw, int &yw) {
  xw = yw = -1;
  if (!P.per_x) xw = (x == 0) ? kLeft : ((x == P.nx - 1) ? kRight : -1);
  if (!P.per_y) yw = (y == 0) ? kBottom : ((y == P.ny - 1) ? kTop : -1);
}

template <class G>
LBS_HD bool on_wall(const G &P, int x, int y) {
  return (!P.per_x && (x == 0 || x == P.nx - 1)) || (!P.per_y && (y == 0 || y == P.ny - 1));
}

// Offset (in values) of the side-array entry of position pos along edge e:
// layer 0 holds N at the wall nodes, layer 1 (two-point wall extrapolation
// only) N at the nodes one step inwards; 4 values per entry, blen entries
// per edge (pos < blen).
template <class G>
LBS_HD size_t side_entry(const G &P, int layer, int e, int pos) {
  return (((size_t)layer * 4 + e) * P.blen + pos) * 4;
}

// The layer-1 entries (two-point wall extrapolation) that node (x, y) fills:
// it is the node one step inwards from each walled edge e[i] at position
// pos[i] along it.  Returns their number (0 to 4; a 3-node axis has one node
// inwards from both of its walls).
template <class G>
LBS_HD int inner_entries(const G &P, int x, int y, int e[4], int pos[4]) {
  int n = 0;
  auto put = [&](int edge, int p) {
    e[n] = edge;
    pos[n] = p;
    ++n;
  };
  if (!P.per_x) {
    if (x == 1) put(kLeft, y);
    if (x == P.nx - 2) put(kRight, y);
  }
  if (!P.per_y) {
    if (y == 1) put(kBottom, x);
    if (y == P.ny - 2) put(kTop, x);
  }
  return n;
}

// the node one step inwards from wall e of wall node (x, y), along its normal
LBS_HD void inner_node(int e, int x, int y, int &xi, int &yi) {
  xi = e == kLeft ? x + 1 : (e == kRight ? x - 1 : x);
  yi = e == kBottom ? y + 1 : (e == kTop ? y - 1 : y);
}

// Finite-difference taps of node (gxn, gyn) (wrapped coordinates) at shared
// position (cx, cy): xa / xb along x and ya / yb along y.  Central inside; on
// the first or last node of a walled axis the node itself replaces the
// outer neighbour (a one-sided difference: onex / oney set).  Without EDGE
// the tile lies clear of the walls and the taps are always central.
template <bool EDGE, class G>
LBS_HD void fd_taps(const G &P, int cx, int cy, int gxn, int gyn, int &xa, int &xb, int &ya, int &yb, bool &onex,
                    bool &oney) {
  xa = cx + 1;
  xb = cx - 1;
  ya = cy + 1;
  yb = cy - 1;
  onex = oney = false;
  if (EDGE) {
    if (!P.per_x) {
      if (gxn == 0) {
        xb = cx;
        onex = true;
      } else if (gxn == P.nx - 1) {
        xa = cx;
        onex = true;
      }
    }
    if (!P.per_y) {
      if (gyn == 0) {
        yb = cy;
        oney = true;
      } else if (gyn == P.ny - 1) {
        ya = cy;
        oney = true;
      }
    }
  }
}

// R1 position (rx, ry) of the tile at (x0, y0) is one of the tile's own
// lattice nodes (not halo, not past the end of the lattice)
template <class C, class G>
LBS_HD bool r1_own_node(const G &P, int x0, int y0, int rx, int ry) {
  return rx >= 1 && rx <= C::TX && ry >= 1 && ry <= C::TY && x0 - 1 + rx < P.nx && y0 - 1 + ry < P.ny;
}

// Interior tile range [a_lo, a_hi) x [b_lo, b_hi) (in tiles): R2 of the tile
// and the streaming sources of R2 (a 3-node frame) stay clear of the walls
// and of the lattice end.  Empty ranges are normalised to (0, 0).
LBS_HD void interior_range(int nx, int ny, int TX, int TY, int &a_lo, int &a_hi, int &b_lo, int &b_hi) {
  a_lo = (3 + TX - 1) / TX;
  a_hi = (nx - 3 - TX) >= 0 ? (nx - 3 - TX) / TX + 1 : 0;
  b_lo = (3 + TY - 1) / TY;
  b_hi = (ny - 3 - TY) >= 0 ? (ny - 3 - TY) / TY + 1 : 0;
  if (a_hi <= a_lo) a_lo = a_hi = 0;
  if (b_hi <= b_lo) b_lo = b_hi = 0;
}

// As interior_range, with the tile's read region reaching `margin` nodes
// beyond it (3 for one iteration, 6 for two fused iterations).
LBS_HD void interior_range_m(int nx, int ny, int TX, int TY, int margin, int &a_lo, int &a_hi, int &b_lo, int &b_hi) {
  a_lo = (margin + TX - 1) / TX;
  a_hi = (nx - margin - TX) >= 0 ? (nx - margin - TX) / TX + 1 : 0;
  b_lo = (margin + TY - 1) / TY;
  b_hi = (ny - margin - TY) >= 0 ? (ny - margin - TY) / TY + 1 : 0;
  if (a_hi <= a_lo) a_lo = a_hi = 0;
  if (b_hi <= b_lo) b_lo = b_hi = 0;
}

// Tile (a, b) of frame tile e: the rows of tiles below the interior block,
// the tiles left and right of it, then the rows above it (ntx tiles per row).
LBS_HD void edge_tile(int e, int ntx, int a_lo, int a_hi, int b_lo, int b_hi, int &a, int &b) {
  const int bottom = ntx * b_lo;
  if (e < bottom) {
    a = e % ntx;
    b = e / ntx;
    return;
  }
  e -= bottom;
  const int side = ntx - (a_hi - a_lo);
  const int mid = side * (b_hi - b_lo);
  if (e < mid) {
    b = b_lo + e / side;
    const int c = e % side;
    a = c < a_lo ? c : a_hi + (c - a_lo);
    return;
  }
  e -= mid;
  a = e % ntx;
  b = b_hi + e / ntx;
}

// ------------------------------------------------------------------ TMA boxes
// Shared-memory layout of a TMA-staged tile (element sizes GS of a stored
// population, US of a displacement record): the nine g planes of the tile
// plus a 3-node halo in a GH x GW box whose first column is node x0 - XO (XO
// rounded up to 16 bytes, so that the box starts on a 16-byte boundary of a
// row), and u on R2 (UH x UW).
template <int TX_, int TY_, int GS, int US>
struct TmaGeom {
  static constexpr int TX = TX_, TY = TY_;
  static constexpr int ALIGN = 16 / GS;                                   // elements per 16 bytes
  static constexpr int XO = ((3 + ALIGN - 1) / ALIGN) * ALIGN;            // box column of node x0
  static constexpr int GW = ((XO + TX + 3 + ALIGN - 1) / ALIGN) * ALIGN;  // box width
  static constexpr int GH = TY + 6;                                       // rows y0-3 .. y0+TY+2
  static constexpr int UW = TX + 4, UH = TY + 4;                          // u on R2
};

// Two fused iterations per launch (temporal blocking): an output tile of TX x
// TY nodes at (x0, y0) advances k -> k + 2 from g_k on the tile plus 6 nodes
// and u_k on the tile plus 5.  Shared arrays, in node offsets (i, j) from
// (x0, y0):
//   g box (GS-byte values, nine planes): j in [-6, TY + 6) (GH rows), i from
//     -XO (XO = 6 rounded up to 16 bytes, so a TMA box starts aligned) over
//     GW columns;
//   u box (US-byte records): i in [-5, TX + 5), j in [-5, TY + 5);
//   g1 (g_{k+1}, GS-byte values, nine planes) on i in [-3, TX + 3), j in [-3, TY + 3);
//   N (four planes) on i in [-4, TX + 4), j in [-4, TY + 4).
template <int TX_, int TY_, int GS, int US>
struct Fuse2Geom {
  static constexpr int TX = TX_, TY = TY_;
  static constexpr int ALIGN = 16 / GS;
  static constexpr int XO = ((6 + ALIGN - 1) / ALIGN) * ALIGN;
  static constexpr int GW = ((XO + TX + 6 + ALIGN - 1) / ALIGN) * ALIGN;
  static constexpr int GH = TY + 12;
  static constexpr int UW = TX + 10, UH = TY + 10;
  static constexpr int HW = TX + 6, HH = TY + 6;
  static constexpr int NW = TX + 8, NH = TY + 8;
  // flat offsets of node offset (i, j) in each array (plane q / m first)
  static LBS_HD int g(int q, int i, int j) { return (q * GH + j + 6) * GW + i + XO; }
  static LBS_HD int u(int i, int j) { return (j + 5) * UW + i + 5; }
  static LBS_HD int h(int q, int i, int j) { return (q * HH + j + 3) * HW + i + 3; }
  static LBS_HD int n(int m, int i, int j) { return (m * NH + j + 4) * NW + i + 4; }
};

}  // namespace lbs
