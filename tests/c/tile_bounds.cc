// Host-side bounds audit of the tiled kernels' index arithmetic.
//
// The kernels take every index from paper_2502_00920_gb300/csrc/lbs_tiles.h
// (tile geometry, ring positions, wrap-around, streaming sources, the links a
// wall rule replaces, finite-difference taps, side-array entries, frame-tile
// enumeration, TMA boxes).  This program includes the same header and walks
// the kernels' loops on the host, for every tile shape the library compiles
// (and the one-node-per-thread frame pieces), over ragged and degenerate
// lattices with every combination of periodic and walled axes and both wall
// readings.  It checks, for one iteration:
//   - every shared-memory index lies in its array, and every shared entry a
//     phase reads was written by an earlier phase of the same tile;
//   - every node a thread updates had its streamed populations gathered
//     (no register of an unvisited node is used);
//   - every global read and write hits a lattice node (never a padding
//     column or a row past the end), and every node is written exactly once
//     per iteration across the interior and frame launches;
//   - the links a wall rule replaces are exactly those whose source lies
//     beyond a wall;
//   - the boundary side array: every entry written lies in the allocation,
//     is written once, and every entry read was written by the previous
//     iteration (or by the initialisation);
//   - the TMA boxes start on 16-byte boundaries and every staged value the
//     kernels use is a lattice node.
// Prints "ok <cases>" and exits 0, or lists the first failures and exits 1.
#include <stdio.h>
#include <stdlib.h>

#include <string>
#include <vector>

#include "lbs_tiles.h"

using namespace lbs;

namespace {

struct Lat {
  int nx, ny, pitch, per_x, per_y, blen, extrap;
};

long g_fail = 0;
std::string g_ctx;

void fail(const char *what, int a = 0, int b = 0, int c = 0) {
  if (g_fail++ < 25) fprintf(stderr, "FAIL [%s] %s (%d, %d, %d)\n", g_ctx.c_str(), what, a, b, c);
}
#define CHECK(cond, ...)          \
  do {                            \
    if (!(cond)) fail(__VA_ARGS__); \
  } while (0)

bool in_lattice(const Lat &P, int x, int y) { return x >= 0 && x < P.nx && y >= 0 && y < P.ny; }

size_t side_values(const Lat &P) { return (size_t)(P.extrap ? 2 : 1) * 4 * P.blen * 4; }

// entries (in units of 4 values) written and read during one iteration
struct Iter {
  std::vector<int> node_w;       // writes of g/u per node
  std::vector<int> side_w;       // writes per side-array entry
  std::vector<char> side_r;      // entries read
  explicit Iter(const Lat &P)
      : node_w((size_t)P.nx * P.ny, 0), side_w(side_values(P) / 4, 0), side_r(side_values(P) / 4, 0) {}
};

void side_write(const Lat &P, Iter &it, int layer, int e, int pos) {
  CHECK(layer == 0 || P.extrap, "side layer 1 without the linear reading", layer, e, pos);
  CHECK(pos >= 0 && pos < ((e == kLeft || e == kRight) ? P.ny : P.nx), "side position beyond its edge", e, pos);
  const size_t o = side_entry(P, layer, e, pos);
  CHECK(o % 4 == 0 && o + 4 <= side_values(P), "side write outside the array", layer, e, pos);
  if (o + 4 <= side_values(P)) it.side_w[o / 4] += 1;
}

void side_read(const Lat &P, Iter &it, int layer, int e, int pos) {
  CHECK(pos >= 0 && pos < ((e == kLeft || e == kRight) ? P.ny : P.nx), "side read beyond its edge", e, pos);
  const size_t o = side_entry(P, layer, e, pos);
  CHECK(o + 4 <= side_values(P), "side read outside the array", layer, e, pos);
  if (o + 4 <= side_values(P)) it.side_r[o / 4] = 1;
}

// gather() of one node (already located): its own populations, the streamed
// ones, and the wall rules' reads (every wall is taken as Neumann, the rule
// that reads the side array)
template <bool EDGE>
void gather(const Lat &P, Iter &it, int x, int y) {
  CHECK(in_lattice(P, x, y), "gather at a node outside the lattice", x, y);
  unsigned mask = 0;
  for (int q = 0; q < 9; ++q) {
    if (!EDGE) {
      CHECK(in_lattice(P, x - ex(q), y - ey(q)), "interior tile streams from outside", x, y, q);
      continue;
    }
    int sx, sy;
    if (stream_source(P, x, y, q, sx, sy)) CHECK(in_lattice(P, sx, sy), "stream source outside", sx, sy, q);
    else mask |= 1u << q;
  }
  if (!mask) return;
  int xw, yw;
  walls_of(P, x, y, xw, yw);
  for (int q = 1; q < 9; ++q) {
    bool ox, oy;
    link_crosses(P, x, y, q, ox, oy);
    CHECK(((mask >> q) & 1) == (unsigned)(ox || oy), "wall rule and streaming disagree on a link", x, y, q);
    CHECK(!ox || xw >= 0, "link crosses an x wall the node is not on", x, y, q);
    CHECK(!oy || yw >= 0, "link crosses a y wall the node is not on", x, y, q);
  }
  if (xw >= 0) side_read(P, it, 0, xw, y);
  if (yw >= 0) side_read(P, it, 0, yw, x);
  if (P.extrap) {
    for (int w = 0; w < 2; ++w) {
      const int e = w == 0 ? xw : yw;
      if (e < 0) continue;
      int xi, yi;
      inner_node(e, x, y, xi, yi);
      CHECK(in_lattice(P, xi, yi), "inner node outside the lattice", xi, yi, e);
      const int pos = w == 0 ? y : x;
      side_read(P, it, 0, e, pos);
      side_read(P, it, 1, e, pos);
    }
  }
}

// one tile of step_tile<C, EDGE, LIN> (the frame and interior kernels, the
// batch kernel's tiles): phases 1a, 1b, 2, 3 over all threads
template <class C, bool EDGE>
void step_tile(const Lat &P, Iter &it, int x0, int y0) {
  std::vector<char> su((size_t)C::R2W * C::R2H, 0), sn((size_t)C::R1W * C::R1H, 0);
  std::vector<char> fset((size_t)C::NT * C::CPT, 0);
  auto su_at = [&](int rx, int ry, bool write, const char *what) {
    if (rx < 0 || rx >= C::R2W || ry < 0 || ry >= C::R2H) {
      fail(what, rx, ry, -2);
      return;
    }
    char &s = su[(size_t)ry * C::R2W + rx];
    if (write) s += 1;
    else CHECK(s == 1, what, rx, ry, s);
  };
  // phase 1a: own nodes
  for (int t = 0; t < C::NT; ++t)
    for (int i = 0; i < C::CPT; ++i) {
      const int lx = t % C::TX, ly = t / C::TX + i * C::NTY;
      int x = x0 + lx, y = y0 + ly;
      if (EDGE && !locate(P, x, y)) continue;
      gather<EDGE>(P, it, x, y);
      su_at(lx + 2, ly + 2, true, "phase 1a writes u outside R2");
      fset[(size_t)t * C::CPT + i] = 1;
    }
  // phase 1b: the 2-node ring
  for (int e = 0; e < C::NRING; ++e) {
    int rx, ry;
    ring_pos<C>(e, rx, ry);
    CHECK(!(rx >= 2 && rx < C::TX + 2 && ry >= 2 && ry < C::TY + 2), "ring entry inside the tile", rx, ry, e);
    int x = x0 - 2 + rx, y = y0 - 2 + ry;
    if (EDGE && !locate(P, x, y)) continue;
    gather<EDGE>(P, it, x, y);
    su_at(rx, ry, true, "phase 1b writes u outside R2");
  }
  for (char s : su) CHECK(s <= 1, "an R2 entry written twice", s);
  // phase 2: N on R1
  for (int e = 0; e < C::R1W * C::R1H; ++e) {
    const int rx = e % C::R1W, ry = e / C::R1W;
    int gx = x0 - 1 + rx, gy = y0 - 1 + ry;
    if (EDGE && !locate(P, gx, gy)) continue;
    CHECK(in_lattice(P, gx, gy), "phase 2 at a node outside the lattice", gx, gy);
    int xa, xb, ya, yb;
    bool onex, oney;
    fd_taps<EDGE>(P, rx + 1, ry + 1, gx, gy, xa, xb, ya, yb, onex, oney);
    su_at(xa, ry + 1, false, "gradient reads an unwritten u (x+)");
    su_at(xb, ry + 1, false, "gradient reads an unwritten u (x-)");
    su_at(rx + 1, ya, false, "gradient reads an unwritten u (y+)");
    su_at(rx + 1, yb, false, "gradient reads an unwritten u (y-)");
    sn[(size_t)ry * C::R1W + rx] = 1;
    if (EDGE && r1_own_node<C>(P, x0, y0, rx, ry)) {
      int xw, yw;
      walls_of(P, gx, gy, xw, yw);
      CHECK(on_wall(P, gx, gy) == (xw >= 0 || yw >= 0), "on_wall and walls_of disagree", gx, gy);
      if (xw >= 0) side_write(P, it, 0, xw, gy);
      if (yw >= 0) side_write(P, it, 0, yw, gx);
      if (P.extrap) {
        int ee[4], pos[4];
        const int n = inner_entries(P, gx, gy, ee, pos);
        for (int k = 0; k < n; ++k) side_write(P, it, 1, ee[k], pos[k]);
      }
    }
  }
  // phase 3: source, collision, stores
  for (int t = 0; t < C::NT; ++t)
    for (int i = 0; i < C::CPT; ++i) {
      const int lx = t % C::TX, ly = t / C::TX + i * C::NTY;
      const int x = x0 + lx, y = y0 + ly;
      if (EDGE && (x >= P.nx || y >= P.ny)) continue;
      CHECK(in_lattice(P, x, y), "phase 3 stores outside the lattice", x, y);
      CHECK(fset[(size_t)t * C::CPT + i] == 1, "phase 3 uses populations never gathered", x, y);
      int xa, xb, ya, yb;
      bool onex, oney;
      fd_taps<EDGE>(P, lx + 1, ly + 1, x, y, xa, xb, ya, yb, onex, oney);
      const int taps[4][2] = {{xa, ly + 1}, {xb, ly + 1}, {lx + 1, ya}, {lx + 1, yb}};
      for (auto &tp : taps) {
        const bool ok = tp[0] >= 0 && tp[0] < C::R1W && tp[1] >= 0 && tp[1] < C::R1H;
        CHECK(ok && sn[(size_t)tp[1] * C::R1W + tp[0]] == 1, "divergence reads an unwritten N", x, y);
      }
      su_at(lx + 2, ly + 2, false, "store reads an unwritten u");
      if (in_lattice(P, x, y)) it.node_w[(size_t)y * P.nx + x] += 1;
    }
}

// one iteration of launch_step<C> (split: the frame tiles as CPT pieces of
// one node per thread)
template <class C>
void launch_step(const Lat &P, Iter &it, bool split) {
  using Piece = TileGeom<C::TX, C::NTY, C::NTY>;
  const int ntx = (P.nx + C::TX - 1) / C::TX, nty = (P.ny + C::TY - 1) / C::TY;
  int a_lo, a_hi, b_lo, b_hi;
  interior_range(P.nx, P.ny, C::TX, C::TY, a_lo, a_hi, b_lo, b_hi);
  const int ni = a_hi - a_lo, nj = b_hi - b_lo;
  for (int b = b_lo; b < b_hi; ++b)
    for (int a = a_lo; a < a_hi; ++a) step_tile<C, false>(P, it, a * C::TX, b * C::TY);
  const int nedge = ntx * nty - ni * nj;
  std::vector<char> seen((size_t)ntx * nty, 0);
  for (int e = 0; e < nedge; ++e) {
    int a, b;
    edge_tile(e, ntx, a_lo, a_hi, b_lo, b_hi, a, b);
    const bool ok = a >= 0 && a < ntx && b >= 0 && b < nty && !(a >= a_lo && a < a_hi && b >= b_lo && b < b_hi);
    CHECK(ok, "frame tile outside the frame", a, b, e);
    if (!ok) continue;
    CHECK(!seen[(size_t)b * ntx + a], "frame tile enumerated twice", a, b);
    seen[(size_t)b * ntx + a] = 1;
    if (split)
      for (int part = 0; part < C::CPT; ++part) step_tile<Piece, true>(P, it, a * C::TX, b * C::TY + part * C::NTY);
    else
      step_tile<C, true>(P, it, a * C::TX, b * C::TY);
  }
}

// the initialisation kernel (and the field-output kernels, which read the
// same R2/R1 entries): every tile loads u on R2, forms N on R1 (writing the
// side array), then reads the taps of its own nodes
template <class C>
void init_fields(const Lat &P, Iter &it) {
  const int ntx = (P.nx + C::TX - 1) / C::TX, nty = (P.ny + C::TY - 1) / C::TY;
  for (int b = 0; b < nty; ++b)
    for (int a = 0; a < ntx; ++a) {
      const int x0 = a * C::TX, y0 = b * C::TY;
      std::vector<char> su((size_t)C::R2W * C::R2H, 0), sn((size_t)C::R1W * C::R1H, 0);
      for (int e = 0; e < C::R2W * C::R2H; ++e) {
        int x = x0 - 2 + e % C::R2W, y = y0 - 2 + e / C::R2W;
        if (locate(P, x, y)) su[e] = 1;
      }
      for (int e = 0; e < C::R1W * C::R1H; ++e) {
        const int rx = e % C::R1W, ry = e / C::R1W;
        int gx = x0 - 1 + rx, gy = y0 - 1 + ry;
        if (!locate(P, gx, gy)) continue;
        int xa, xb, ya, yb;
        bool onex, oney;
        fd_taps<true>(P, rx + 1, ry + 1, gx, gy, xa, xb, ya, yb, onex, oney);
        CHECK(su[(size_t)(ry + 1) * C::R2W + xa] && su[(size_t)(ry + 1) * C::R2W + xb] &&
                  su[(size_t)ya * C::R2W + rx + 1] && su[(size_t)yb * C::R2W + rx + 1],
              "initial gradient reads an unloaded u", gx, gy);
        sn[e] = 1;
        if (r1_own_node<C>(P, x0, y0, rx, ry)) {
          int xw, yw;
          walls_of(P, gx, gy, xw, yw);
          if (xw >= 0) side_write(P, it, 0, xw, gy);
          if (yw >= 0) side_write(P, it, 0, yw, gx);
          if (P.extrap) {
            int ee[4], pos[4];
            const int n = inner_entries(P, gx, gy, ee, pos);
            for (int k = 0; k < n; ++k) side_write(P, it, 1, ee[k], pos[k]);
          }
        }
      }
      for (int t = 0; t < C::NT; ++t)
        for (int i = 0; i < C::CPT; ++i) {
          const int lx = t % C::TX, ly = t / C::TX + i * C::NTY, x = x0 + lx, y = y0 + ly;
          if (x >= P.nx || y >= P.ny) continue;
          int xa, xb, ya, yb;
          bool onex, oney;
          fd_taps<true>(P, lx + 1, ly + 1, x, y, xa, xb, ya, yb, onex, oney);
          CHECK(sn[(size_t)(ly + 1) * C::R1W + xa] && sn[(size_t)(ly + 1) * C::R1W + xb] &&
                    sn[(size_t)ya * C::R1W + lx + 1] && sn[(size_t)yb * C::R1W + lx + 1],
                "initial divergence reads an unwritten N", x, y);
          it.node_w[(size_t)y * P.nx + x] += 1;
        }
    }
}

// every node once; side entries written once each, exactly the wall-node
// (and, with the linear reading, inner-node) entries; reads within the writes
void check_iteration(const Lat &P, const Iter &it, const Iter &prev_writes, const char *what) {
  for (int y = 0; y < P.ny; ++y)
    for (int x = 0; x < P.nx; ++x)
      CHECK(it.node_w[(size_t)y * P.nx + x] == 1, what, x, y, it.node_w[(size_t)y * P.nx + x]);
  std::vector<int> want(it.side_w.size(), 0);
  for (int y = 0; y < P.ny; ++y)
    for (int x = 0; x < P.nx; ++x) {
      int xw, yw;
      walls_of(P, x, y, xw, yw);
      if (xw >= 0) want[side_entry(P, 0, xw, y) / 4] += 1;
      if (yw >= 0) want[side_entry(P, 0, yw, x) / 4] += 1;
      if (P.extrap) {
        int ee[4], pos[4];
        const int n = inner_entries(P, x, y, ee, pos);
        for (int k = 0; k < n; ++k) want[side_entry(P, 1, ee[k], pos[k]) / 4] += 1;
      }
    }
  for (size_t i = 0; i < want.size(); ++i) {
    CHECK(want[i] <= 1, "two nodes own one side entry", (int)i);
    CHECK(it.side_w[i] == want[i], "side entry written a wrong number of times", (int)i, it.side_w[i], want[i]);
    CHECK(!it.side_r[i] || prev_writes.side_w[i] == 1, "side entry read but not written before", (int)i);
  }
}

// TMA-staged interior tiles (step_tma_kernel, step_tma2_kernel): box origins
// on 16-byte boundaries, every staged value used lies in the lattice
template <int TX, int TY, int NTY, int GS, int US>
void check_tma(const Lat &P, Iter &it) {
  using T = TmaGeom<TX, TY, GS, US>;
  int a_lo, a_hi, b_lo, b_hi;
  interior_range(P.nx, P.ny, TX, TY, a_lo, a_hi, b_lo, b_hi);
  for (int b = b_lo; b < b_hi; ++b)
    for (int a = a_lo; a < a_hi; ++a) {
      const int x0 = a * TX, y0 = b * TY;
      const long gx_bytes = (long)(x0 - T::XO) * GS, ux_bytes = (long)(x0 - 2) * US;
      CHECK(gx_bytes % 16 == 0 && ux_bytes % 16 == 0, "TMA box not on a 16-byte boundary", x0, y0);
      CHECK(T::GW * GS % 16 == 0, "TMA g box width not a multiple of 16 bytes", T::GW);
      auto g_used = [&](int r, int c) {
        CHECK(r >= 0 && r < T::GH && c >= 0 && c < T::GW, "g box index outside the box", r, c);
        CHECK(in_lattice(P, x0 - T::XO + c, y0 - 3 + r), "staged g value used outside the lattice", x0, y0);
      };
      for (int cy = 0; cy < T::UH; ++cy)
        for (int cx = 0; cx < T::UW; ++cx) {
          CHECK(in_lattice(P, x0 - 2 + cx, y0 - 2 + cy), "staged u outside the lattice", cx, cy);
          for (int q = 1; q < 9; ++q) {
            g_used(cy + 1 - ey(q), cx + T::XO - 2 - ex(q));
            g_used(cy + 1, cx + T::XO - 2);
          }
        }
      for (int ry = 0; ry < TY + 2; ++ry)
        for (int rx = 0; rx < TX + 2; ++rx) {
          const int c = (ry + 1) * T::UW + (rx + 1);
          CHECK(c - T::UW >= 0 && c + T::UW < T::UW * T::UH, "u taps outside the staged box", rx, ry);
        }
      for (int t = 0; t < TX * NTY; ++t)
        for (int i = 0; i < TY / NTY; ++i) {
          const int lx = t % TX, ly = t / TX + i * NTY;
          for (int q = 0; q < 9; ++q) g_used(ly + 3 - ey(q), lx + T::XO - ex(q));
          it.node_w[(size_t)(y0 + ly) * P.nx + x0 + lx] += 1;
        }
    }
}

// frame kernel of the TMA variants: launch_step's frame tiles
template <class C>
void frame_only(const Lat &P, Iter &it, bool split) {
  using Piece = TileGeom<C::TX, C::NTY, C::NTY>;
  const int ntx = (P.nx + C::TX - 1) / C::TX, nty = (P.ny + C::TY - 1) / C::TY;
  int a_lo, a_hi, b_lo, b_hi;
  interior_range(P.nx, P.ny, C::TX, C::TY, a_lo, a_hi, b_lo, b_hi);
  const int nedge = ntx * nty - (a_hi - a_lo) * (b_hi - b_lo);
  for (int e = 0; e < nedge; ++e) {
    int a, b;
    edge_tile(e, ntx, a_lo, a_hi, b_lo, b_hi, a, b);
    if (split)
      for (int part = 0; part < C::CPT; ++part) step_tile<Piece, true>(P, it, a * C::TX, b * C::TY + part * C::NTY);
    else
      step_tile<C, true>(P, it, a * C::TX, b * C::TY);
  }
}

// two fused iterations (periodic lattices): interior tiles staged by TMA
// (boxes aligned, every staged value used a lattice node), frame tiles
// gathered with wrapped loads; every array index within its array, every
// node stored once per call
template <int TX, int TY, int NTY, int GS, int US>
void check_fused2(const Lat &P, Iter &it) {
  using F = Fuse2Geom<TX, TY, GS, US>;
  const int ntx = (P.nx + TX - 1) / TX, nty = (P.ny + TY - 1) / TY;
  int a_lo, a_hi, b_lo, b_hi;
  interior_range_m(P.nx, P.ny, TX, TY, 6, a_lo, a_hi, b_lo, b_hi);
  auto tile = [&](int x0, int y0, bool tma) {
    if (tma) {
      CHECK((long)(x0 - F::XO) * GS % 16 == 0 && (long)(x0 - 5) * US % 16 == 0, "fused TMA box misaligned", x0, y0);
      CHECK(F::GW * GS % 16 == 0, "fused g box width not a multiple of 16 bytes", F::GW);
    }
    auto g_at = [&](int q, int i, int j) {
      const int o = F::g(q, i, j);
      CHECK(o >= 0 && o < 9 * F::GH * F::GW && i + F::XO >= 0 && i + F::XO < F::GW, "fused g index", i, j, q);
      int x = x0 + i, y = y0 + j;
      if (tma) CHECK(in_lattice(P, x, y), "fused TMA value used outside the lattice", x, y);
      else CHECK(locate(P, x, y) && in_lattice(P, x, y), "fused frame value does not wrap into the lattice", x, y);
    };
    auto u_at = [&](int i, int j) {
      const int o = F::u(i, j);
      CHECK(o >= 0 && o < F::UW * F::UH && i >= -5 && i < TX + 5 && j >= -5 && j < TY + 5, "fused u index", i, j);
    };
    auto h_at = [&](int q, int i, int j) {
      CHECK(i >= -3 && i < TX + 3 && j >= -3 && j < TY + 3 && F::h(q, i, j) < 9 * F::HW * F::HH, "fused g1 index", i,
            j, q);
    };
    auto n_at = [&](int m, int i, int j) {
      CHECK(i >= -4 && i < TX + 4 && j >= -4 && j < TY + 4 && F::n(m, i, j) < 4 * F::NW * F::NH, "fused N index", i,
            j, m);
    };
    for (int j = -5; j < TY + 5; ++j)  // u_{k+1} on tile + 5
      for (int i = -5; i < TX + 5; ++i) {
        u_at(i, j);
        for (int q = 1; q < 9; ++q) g_at(q, i - ex(q), j - ey(q));
      }
    for (int j = -4; j < TY + 4; ++j)  // N on tile + 4
      for (int i = -4; i < TX + 4; ++i) {
        u_at(i + 1, j), u_at(i - 1, j), u_at(i, j + 1), u_at(i, j - 1);
        n_at(0, i, j);
      }
    for (int j = -3; j < TY + 3; ++j)  // g_{k+1} on tile + 3
      for (int i = -3; i < TX + 3; ++i) {
        for (int q = 0; q < 9; ++q) g_at(q, i - ex(q), j - ey(q)), h_at(q, i, j);
        n_at(1, i + 1, j), n_at(1, i - 1, j), n_at(1, i, j + 1), n_at(1, i, j - 1);
      }
    for (int j = -2; j < TY + 2; ++j)  // u_{k+2} on tile + 2
      for (int i = -2; i < TX + 2; ++i)
        for (int q = 1; q < 9; ++q) h_at(q, i - ex(q), j - ey(q));
    for (int j = -1; j < TY + 1; ++j)  // N on tile + 1
      for (int i = -1; i < TX + 1; ++i) n_at(2, i, j);
    for (int t = 0; t < TX * NTY; ++t)  // g_{k+2} on the tile
      for (int c = 0; c < TY / NTY; ++c) {
        const int i = t % TX, j = t / TX + c * NTY;
        for (int q = 0; q < 9; ++q) h_at(q, i - ex(q), j - ey(q));
        const int x = x0 + i, y = y0 + j;
        if (x < P.nx && y < P.ny) it.node_w[(size_t)y * P.nx + x] += 1;
      }
  };
  for (int b = b_lo; b < b_hi; ++b)
    for (int a = a_lo; a < a_hi; ++a) tile(a * TX, b * TY, true);
  const int nedge = ntx * nty - (a_hi - a_lo) * (b_hi - b_lo);
  for (int e = 0; e < nedge; ++e) {
    int a, b;
    edge_tile(e, ntx, a_lo, a_hi, b_lo, b_hi, a, b);
    tile(a * TX, b * TY, false);
  }
}

long g_cases = 0;

template <int TX, int TY, int NTY>
void shape_cases(const std::vector<int> &sizes) {
  using C = TileGeom<TX, TY, NTY>;
  for (int nx : sizes)
    for (int ny : sizes)
      for (int per = 0; per < 4; ++per)
        for (int extrap = 0; extrap < 2; ++extrap) {
          Lat P{nx, ny, (nx + 31) / 32 * 32, per & 1, (per >> 1) & 1, nx > ny ? nx : ny, extrap};
          char buf[160];
          snprintf(buf, sizeof buf, "tile %dx%d/%d, lattice %dx%d, periodic x %d y %d, linear %d", TX, TY, NTY, nx, ny,
                   P.per_x, P.per_y, extrap);
          g_ctx = buf;
          Iter init(P);
          init_fields<TileGeom<32, 16, 8>>(P, init);
          check_iteration(P, init, init, "initialisation writes each node once");
          for (int split = 0; split < (C::CPT > 1 ? 2 : 1); ++split) {
            Iter it(P);
            launch_step<C>(P, it, split);
            check_iteration(P, it, init, "a step writes each node once");
            Iter it2(P);
            launch_step<C>(P, it2, split);
            check_iteration(P, it2, it, "a second step writes each node once");
            ++g_cases;
          }
        }
}

template <int TX, int TY, int NTY, int GS, int US>
void tma_cases(const std::vector<int> &sizes) {
  using C = TileGeom<TX, TY, NTY>;
  for (int nx : sizes)
    for (int ny : sizes)
      for (int per = 0; per < 4; ++per) {
        Lat P{nx, ny, (nx + 31) / 32 * 32, per & 1, (per >> 1) & 1, nx > ny ? nx : ny, 0};
        char buf[160];
        snprintf(buf, sizeof buf, "TMA tile %dx%d/%d (%d-byte g), lattice %dx%d, periodic x %d y %d", TX, TY, NTY, GS,
                 nx, ny, P.per_x, P.per_y);
        g_ctx = buf;
        Iter init(P);
        init_fields<TileGeom<32, 16, 8>>(P, init);
        for (int split = 0; split < (C::CPT > 1 ? 2 : 1); ++split) {
          Iter it(P);
          check_tma<TX, TY, NTY, GS, US>(P, it);
          frame_only<C>(P, it, split);
          check_iteration(P, it, init, "a TMA step writes each node once");
          ++g_cases;
        }
      }
}

template <int TX, int TY, int NTY, int GS, int US>
void fused2_cases(const std::vector<int> &sizes) {
  for (int nx : sizes)
    for (int ny : sizes) {
      if (nx < 16 || ny < 16) continue;  // the fused iterations apply from 16 nodes per axis
      Lat P{nx, ny, (nx + 31) / 32 * 32, 1, 1, nx > ny ? nx : ny, 0};
      char buf[160];
      snprintf(buf, sizeof buf, "fused tile %dx%d/%d (%d-byte g), periodic lattice %dx%d", TX, TY, NTY, GS, nx, ny);
      g_ctx = buf;
      Iter it(P);
      check_fused2<TX, TY, NTY, GS, US>(P, it);
      check_iteration(P, it, it, "a fused call writes each node once");
      ++g_cases;
    }
}

}  // namespace

int main() {
  // ragged and degenerate sizes around the tile widths (32, 64) and heights
  const std::vector<int> small = {3, 4, 5, 7, 8, 9, 15, 16, 17, 23, 24, 25, 31, 32, 33, 35, 36, 37, 40, 63, 64, 65,
                                  67, 70, 71, 97, 100, 131};
  // global-memory tiles of every precision (32x16, 32x8, 64x8 / 4 rows,
  // 32x24, 32x32), their frame pieces, and the batch kernel's 32x16 tiles
  shape_cases<32, 16, 8>(small);
  shape_cases<32, 8, 8>(small);
  shape_cases<64, 8, 4>(small);
  shape_cases<32, 24, 8>(small);
  shape_cases<32, 32, 8>(small);
  // TMA variants: FP64 32x8 (8-byte g, 16-byte u), FP32 32x16 and 32x24
  // (4-byte g), FP16 32x16 and 32x32 (2-byte g); u records are 16 bytes
  tma_cases<32, 8, 8, 8, 16>(small);
  tma_cases<32, 16, 8, 4, 16>(small);
  tma_cases<32, 24, 8, 4, 16>(small);
  tma_cases<32, 16, 8, 2, 16>(small);
  tma_cases<32, 32, 8, 2, 16>(small);
  // two fused iterations: FP32 32x16 tiles, one node per thread
  fused2_cases<32, 16, 16, 4, 16>(small);
  if (g_fail) {
    fprintf(stderr, "%ld failures\n", g_fail);
    return 1;
  }
  printf("ok %ld\n", g_cases);
  return 0;
}
