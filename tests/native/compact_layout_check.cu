// Host-side check of the compacted lattice (no GPU needed): the library's
// own build_host_case + build_compact, then the node word's neighbour rows
// and compact_targets against the dense neighbourhood for
// every fluid node and direction, and pull_slots (where the step kernels
// gather and the conversions scatter) against the same neighbourhood and
// the link table: every slot in range and held by exactly one (node,
// direction); the f_jb slot of every link.
// Geometries: walled and periodic channels, a periodic box, 1-wide
// lattices, random cylinders on every combination of periodic axes, and
// any lattices given as files (int32 nx, ny, periodic_x, periodic_y, then
// nx*ny solid bytes).
#include <cstdio>
#include <cstdlib>
#include <random>
#include <string>
#include <vector>
#include "lbm_internal.h"
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
int check(const char *name, int nx, int ny, int px, int py, std::vector<uint8_t> solid) {
  std::vector<int32_t> lx, ly, ld;
  std::vector<double> q, ub;
  auto wrapok = [&](int x, int y, int &xx, int &yy) {
    xx = x; yy = y;
    if (xx < 0 || xx >= nx) { if (!px) return false; xx = (xx + nx) % nx; }
    if (yy < 0 || yy >= ny) { if (!py) return false; yy = (yy + ny) % ny; }
    return true;
  };
  for (int y = 0; y < ny; y++)
    for (int x = 0; x < nx; x++) {
      if (solid[y * nx + x]) continue;
      for (int i = 1; i < 9; i++) {
        int xx, yy;
        if (!wrapok(x - CX[i], y - CY[i], xx, yy) || solid[yy * nx + xx]) {
          lx.push_back(x); ly.push_back(y); ld.push_back(i); q.push_back(0.5); ub.push_back(0.0);
        }
      }
    }
  lbm_domain_t dom{};
  dom.nx = nx; dom.ny = ny; dom.periodic_x = px; dom.periodic_y = py; dom.H = 10.0; dom.ax = 1e-6; dom.ay = 0;
  lbm_params_t p;
  lbm_params_default(&p);
  lbm::HostCase hc;
  std::string err;
  int rc = lbm::build_host_case(&dom, solid.data(), lx.size(), lx.data(), ly.data(), ld.data(), q.data(),
                                ub.data(), ub.data(), 0.05, &p, &hc, &err);
  if (rc) { printf("%s: build_host_case failed: %s\n", name, err.c_str()); return 1; }
  lbm::CompactCase cc;
  const std::string cerr = lbm::build_compact(hc, &cc);
  if (!cerr.empty()) { printf("%s: build_compact failed: %s\n", name, cerr.c_str()); return 1; }
  long bad = 0, checked = 0;
  const uint32_t P = (uint32_t)cc.plane;
  const std::vector<uint32_t> jbs = lbm::link_jb_slots(cc, ny, py, hc.n_links);
  if ((int64_t)jbs.size() != hc.n_links) bad++;
  const std::vector<uint16_t> lds = lbm::link_descriptors(cc, hc.n_links);
  if ((int64_t)lds.size() != hc.n_links) bad++;
  const uint64_t n_slots = 9ull * P + (uint64_t)hc.n_links;
  std::vector<uint8_t> slot_use(n_slots, 0);
  if (cc.grp.size() != (size_t)((cc.n_fluid + lbm::kGroup - 1) / lbm::kGroup)) bad++;
  for (int y = 0; y < ny; y++)
    for (int x = 0; x < nx; x++) {
      int32_t i = cc.index[y * nx + x];
      if (i < 0) continue;
      // decode the 8-byte node word as the kernel does
      const uint2 nw = cc.node[i];
      uint32_t nb, sb;
      lbm::neighbour_rows(nw, (uint32_t)i, (uint32_t)cc.n_fluid, y, ny, py, nb, sb);
      // n_lb / s_lb by definition: first fluid node at or after (x, y +- 1)
      {
        const int yn = lbm::row_above(y, ny, py), ys = lbm::row_below(y, ny, py);
        int32_t wn = cc.rowstart[yn + 1], ws = cc.rowstart[ys + 1];
        for (int xx = nx - 1; xx >= x; xx--) {
          if (cc.index[yn * nx + xx] >= 0) wn = cc.index[yn * nx + xx];
          if (cc.index[ys * nx + xx] >= 0) ws = cc.index[ys * nx + xx];
        }
        if (nb != (uint32_t)wn || sb != (uint32_t)ws) bad++;
        if ((nw.x >> 16) > (uint32_t)nx || (nw.y & 0xFFFFu) > (uint32_t)nx) bad++;
      }
      uint32_t tq[9];
      lbm::compact_targets(nw.x & lbm::kNodeMeta, i, nb, sb, y, ny, py, cc.rowstart.data(), tq);
      uint8_t fl = nw.x & 0xFF;
      // row and first link from the group record and the node word's offsets
      const int2 gr = cc.grp[i / lbm::kGroup];
      if (gr.x + lbm::node_dy(nw) != y) bad++;
      if (fl && gr.y + (int32_t)lbm::node_loff(nw) != hc.lbase[(size_t)y * hc.pitch + x]) bad++;
      uint32_t ps[9];
      lbm::pull_slots(nw, gr, i, P, (uint32_t)cc.n_fluid, ny, py, cc.rowstart.data(), ps);
      if (ps[0] != (uint32_t)i) bad++;
      int rank = 0;
      for (int qd = 0; qd < 9; qd++) {
        if (ps[qd] >= n_slots) { bad++; continue; }
        if (slot_use[ps[qd]]++) bad++;  // two (node, direction) pairs share a slot
        if (qd == 0) continue;
        int xs, ys;
        const bool src_in = wrapok(x - CX[qd], y - CY[qd], xs, ys);
        const bool src_fluid = src_in && !solid[ys * nx + xs];
        if (src_fluid) {
          if (fl & (1u << (qd - 1))) bad++;
          if (ps[qd] != (uint32_t)qd * P + (uint32_t)cc.index[ys * nx + xs]) {
            if (bad < 5) printf("%s: node (%d,%d) gather %d got %u\n", name, x, y, qd, ps[qd]);
            bad++;
          }
        } else {
          if (!(fl & (1u << (qd - 1)))) bad++;
          // the link of (x, y, qd) in the table, in direction order within the node
          const int64_t link = hc.lbase[(size_t)y * hc.pitch + x] + rank;
          if (ps[qd] != 9u * P + (uint32_t)link) bad++;
          // the link's f_jb slot: x + c_qd if fluid, else the tail slot of link (x, opp(qd))
          int xo, yo;
          const bool opp_in = wrapok(x + CX[qd], y + CY[qd], xo, yo);
          uint32_t want_jb;
          if (opp_in && !solid[yo * nx + xo]) {
            want_jb = (uint32_t)OPP[qd] * P + (uint32_t)cc.index[yo * nx + xo];
          } else {
            const int ob = OPP[qd];
            want_jb = 9u * P + (uint32_t)(hc.lbase[(size_t)y * hc.pitch + x] +
                                          __builtin_popcount(fl & ((1u << (ob - 1)) - 1u)));
          }
          if (jbs[link] != want_jb) bad++;
          // the link's descriptor: its node's place in the node's 64-aligned
          // block and its direction
          if (lds[link] != (uint16_t)(((uint32_t)i & 63u) << 4 | (uint32_t)qd)) bad++;
          rank++;
        }
      }
      if (fl != hc.flags[(size_t)y * hc.pitch + x]) bad++;
      const bool we = px && x == nx - 1, ww = px && x == 0;
      if (((nw.x & lbm::kMetaWrapE) != 0) != we || ((nw.x & lbm::kMetaWrapW) != 0) != ww) bad++;
      for (int qd = 1; qd < 9; qd++) {
        bool fluid_target = !(fl & (1u << (OPP[qd] - 1)));
        int xx, yy;
        bool in = wrapok(x + CX[qd], y + CY[qd], xx, yy);
        bool truth_fluid = in && !solid[yy * nx + xx];
        if (fluid_target != truth_fluid) { bad++; continue; }
        if (!fluid_target) continue;
        checked++;
        int32_t want = cc.index[yy * nx + xx];
        if (tq[qd] != (uint32_t)want || tq[qd] >= (uint32_t)cc.n_fluid) {
          if (bad < 5) printf("%s: node (%d,%d) dir %d got %u want %d\n", name, x, y, qd, tq[qd], want);
          bad++;
        }
      }
      if (cc.lbase[i] != (fl ? hc.lbase[(size_t)y * hc.pitch + x] : 0)) bad++;
    }
  // every link's tail slot is used (by its own node and direction)
  for (uint64_t t = 9ull * P; t < n_slots; t++)
    if (slot_use[t] != 1) bad++;
  printf("%-22s nx %5d ny %5d px %d py %d fluid %8lld links %8lld checked %9ld bad %ld\n", name, nx, ny,
         px, py, (long long)cc.n_fluid, (long long)hc.n_links, checked, bad);
  return bad != 0;
}
int main(int argc, char **argv) {
  int fails = 0;
  auto channel = [](int nx, int ny) { std::vector<uint8_t> s(nx * ny, 0); for (int x = 0; x < nx; x++) { s[x] = 1; s[(ny - 1) * nx + x] = 1; } return s; };
  fails += check("channel", 4, 34, 1, 0, channel(4, 34));
  fails += check("channel_wide", 37, 9, 1, 0, channel(37, 9));
  fails += check("box", 70, 45, 1, 1, std::vector<uint8_t>(70 * 45, 0));
  fails += check("column", 1, 7, 1, 1, std::vector<uint8_t>(7, 0));
  fails += check("row", 33, 1, 1, 1, std::vector<uint8_t>(33, 0));
  fails += check("row_wall_x", 40, 20, 0, 1, [] { std::vector<uint8_t> s(40 * 20, 0); for (int y = 0; y < 20; y++) { s[y * 40] = 1; s[y * 40 + 39] = 1; } return s; }());
  // periodic y with solid blocks at the ends of the last and first rows: the
  // first fluid node at or after (x, y +- 1) is then past the end of that
  // row (for the last row, the end of the lattice)
  // fully solid rows inside a periodic lattice (compact rows skip them)
  fails += check("solid_bands", 30, 12, 1, 1, [] { std::vector<uint8_t> s(30 * 12, 0); for (int x = 0; x < 30; x++) { s[x] = 1; s[5 * 30 + x] = 1; s[6 * 30 + x] = 1; } s[11 * 30 + 7] = 1; s[4 * 30 + 29] = 1; return s; }());
  fails += check("edge_row_gaps", 24, 9, 1, 1, [] { std::vector<uint8_t> s(24 * 9, 0); for (int x = 16; x < 24; x++) { s[8 * 24 + x] = 1; s[x - 16] = 1; } s[4 * 24 + 23] = 1; return s; }());
  std::mt19937 rng(3);
  for (int t = 0; t < 6; t++) {
    int nx = 50 + rng() % 700, ny = 40 + rng() % 300;
    int px = t % 2, py = (t / 2) % 2;
    std::vector<uint8_t> s(nx * ny, 0);
    for (int c = 0; c < nx * ny / 300; c++) {
      int cx = rng() % nx, cy = rng() % ny, r = 2 + rng() % 9;
      for (int y = cy - r; y <= cy + r; y++)
        for (int x = cx - r; x <= cx + r; x++) {
          int xx = ((x % nx) + nx) % nx, yy = ((y % ny) + ny) % ny;
          if ((x - cx) * (x - cx) + (y - cy) * (y - cy) <= r * r) s[yy * nx + xx] = 1;
        }
    }
    if (!px) for (int y = 0; y < ny; y++) { s[y * nx] = 1; s[y * nx + nx - 1] = 1; }
    if (!py) for (int x = 0; x < nx; x++) { s[x] = 1; s[(ny - 1) * nx + x] = 1; }
    // drop fluid nodes enclosed on all sides (the library rejects them)
    for (int y = 0; y < ny; y++) for (int x = 0; x < nx; x++) {
      if (s[y * nx + x]) continue;
      int open = 0;
      for (int i = 1; i < 9; i++) { int xx = x - CX[i], yy = y - CY[i];
        if (xx < 0 || xx >= nx) { if (!px) continue; xx = (xx + nx) % nx; }
        if (yy < 0 || yy >= ny) { if (!py) continue; yy = (yy + ny) % ny; }
        if (!s[yy * nx + xx]) open++; }
      if (!open) s[y * nx + x] = 1;
    }
    char nm[64]; snprintf(nm, sizeof nm, "cylinders_%d", t);
    fails += check(nm, nx, ny, px, py, s);
  }
  for (int a = 1; a < argc; a++) {
    const char *fn = argv[a];
    FILE *f = fopen(fn, "rb");
    if (!f) { printf("%s: cannot open\n", fn); fails++; continue; }
    int32_t hd[4];
    if (fread(hd, 4, 4, f) != 4) return 2;
    std::vector<uint8_t> s((size_t)hd[0] * hd[1]);
    if (fread(s.data(), 1, s.size(), f) != s.size()) return 2;
    fclose(f);
    fails += check(fn, hd[0], hd[1], hd[2], hd[3], s);
  }
  printf(fails ? "FAILED\n" : "ALL OK\n");
  return fails != 0;
}
