// Host lattice builder: voxel labels -> compacted sites, 18-link neighbour
// table, wall-site list, tile descriptors and boundary slot arrays.
//
// The paper's solver is built for "complex and sparse geometries" (Sec. 1);
// it does not describe its data structure, so this one is designed for the
// GPU: sites keep the canonical z-fastest order (so that a warp of 32
// consecutive sites touches contiguous memory along a vessel), and every tile
// of 32 sites is classified once:
//   bulk      all 18 links fluid and, per direction, the same neighbour offset
//             for every lane -> 18 offsets describe the whole tile;
//   coherent  some links leave the fluid, but in every direction the lanes
//             whose link is fluid share one offset (a straight wall column,
//             or a tile at an inlet/outlet plane) -> 18 offsets per tile plus
//             per-site masks saying which links are wall or iolet links;
//   irregular anything else -> per-site link codes.
// Uniform and irregular tiles are the boundary tiles; their per-site data
// (link masks, wall parameters, inlet profile) live in "slots", 32 per tile.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <limits>
#include <thread>
#include <vector>

#include "d3q19.h"
#include "lbm_internal.h"

namespace lbm {

using cplx = std::complex<double>;

namespace {

// Bessel J0 and J1 of complex argument from their integral representations
//   J0(z) = (1/pi) int_0^pi cos(z sin t) dt,  J1(z) = (1/pi) int_0^pi cos(t - z sin t) dt,
// by the trapezoidal rule, which converges geometrically for these periodic
// integrands (error below 1e-13 for |z| <= 25 with 160 panels).
void bessel01(cplx z, cplx& j0, cplx& j1) {
  const int n = 160;
  const double h = M_PI / n;
  cplx s0 = 0.5 * (std::cos(z * 0.0) + std::cos(z * std::sin(M_PI)));
  cplx s1 = 0.5 * (std::cos(cplx(0.0) - z * 0.0) + std::cos(cplx(M_PI) - z * std::sin(M_PI)));
  for (int k = 1; k < n; ++k) {
    const double t = k * h;
    s0 += std::cos(z * std::sin(t));
    s1 += std::cos(cplx(t) - z * std::sin(t));
  }
  j0 = s0 * h / M_PI;
  j1 = s1 * h / M_PI;
}

// Oscillatory axial velocity of rigid-tube Womersley flow (Sec. 2.2 with
// M = 1, c -> infinity) normalised to unit mean over the disc:
//   s(xi) = (1 - J0(L xi)/J0(L)) / (1 - 2 J1(L)/(L J0(L))),  L = i^(3/2) alpha.
cplx womersley(double alpha, double xi) {
  if (alpha < 1e-6) return cplx(2.0 * (1.0 - xi * xi), 0.0);
  const cplx lam = alpha * std::exp(cplx(0.0, 0.75 * M_PI));
  cplx j0L, j1L, j0r, j1r;
  bessel01(lam, j0L, j1L);
  bessel01(lam * xi, j0r, j1r);
  return (1.0 - j0r / j0L) / (1.0 - 2.0 * j1L / (lam * j0L));
}

// Host threads of the builder (the machine's, at most 64).
int host_threads() {
  const unsigned h = std::thread::hardware_concurrency();
  return (int)std::max(1u, std::min(h, 64u));
}

// f(begin, end, thread) over a static split of [0, n) into contiguous ranges,
// in increasing order of thread index; small ranges run on the caller.
template <class F>
void parallel_for(int64_t n, F&& f) {
  const int64_t grain = 1 << 14;
  const int nt = (int)std::min<int64_t>(host_threads(), (n + grain - 1) / grain);
  if (nt <= 1) {
    if (n > 0) f(int64_t(0), n, 0);
    return;
  }
  std::vector<std::thread> th;
  th.reserve(nt);
  for (int t = 0; t < nt; ++t) th.emplace_back([&f, n, nt, t] { f(n * t / nt, n * (t + 1) / nt, t); });
  for (auto& x : th) x.join();
}

bool finite3(const double* v) {
  return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]);
}

}  // namespace

int build_lattice(const uint8_t* labels, int32_t nx, int32_t ny, int32_t nz,
                  const lbm_iolet* iolets, int32_t n_iolets, double tau, HostLattice& L,
                  std::string& err) {
  char msg[256];
  if (nx <= 0 || ny <= 0 || nz <= 0 || n_iolets < 0 || n_iolets > 253 || !labels ||
      (n_iolets > 0 && !iolets)) {
    err = "bad lattice dimensions, iolet count or null pointer";
    return LBM_EINVAL;
  }
  if (!(tau > 0.5) || !std::isfinite(tau)) {
    err = "tau must be finite and > 1/2";
    return LBM_EINVAL;
  }
  for (int k = 0; k < n_iolets; ++k) {
    const lbm_iolet& io = iolets[k];
    const double an = std::sqrt(io.axis[0] * io.axis[0] + io.axis[1] * io.axis[1] +
                                io.axis[2] * io.axis[2]);
    bool ok = (io.kind == LBM_IOLET_VELOCITY || io.kind == LBM_IOLET_DENSITY) &&
              (io.profile >= LBM_PROFILE_PARABOLIC && io.profile <= LBM_PROFILE_PLUG) &&
              an > 0.0 && std::isfinite(an) && finite3(io.centre) && std::isfinite(io.rho) &&
              std::isfinite(io.u_mean) && std::isfinite(io.u_amp) && std::isfinite(io.period) &&
              std::isfinite(io.phase) && std::isfinite(io.radius);
    if (ok && io.kind == LBM_IOLET_VELOCITY && io.profile != LBM_PROFILE_PLUG)
      ok = io.radius > 0.0;
    if (ok && io.kind == LBM_IOLET_DENSITY) ok = io.rho > 0.0;
    if (!ok) {
      std::snprintf(msg, sizeof msg, "iolet %d: bad kind, profile, axis, radius or value", k);
      err = msg;
      return LBM_EINVAL;
    }
  }
  const int max_label = 1 + n_iolets;
  // ---- fluid runs along z, column by column (column c = x ny + y): the site
  // of a fluid voxel is found from its column's runs, so no per-voxel index
  // of the (possibly mostly solid) bounding box is held.
  const int64_t C = (int64_t)nx * ny;
  const int nthr = host_threads();
  std::vector<int32_t> col_n(C), col_runs(C);
  std::vector<int64_t> bad(nthr, std::numeric_limits<int64_t>::max());
  parallel_for(C, [&](int64_t c0, int64_t c1, int t) {
    for (int64_t c = c0; c < c1; ++c) {
      const uint8_t* lab = labels + c * nz;
      int32_t cnt = 0, runs = 0;
      bool in = false;
      for (int32_t z = 0; z < nz; ++z) {
        const int v = lab[z];
        if (v > max_label && bad[t] == std::numeric_limits<int64_t>::max()) bad[t] = c * nz + z;
        const bool f = v == 1;
        cnt += f;
        runs += (f && !in);
        in = f;
      }
      col_n[c] = cnt;
      col_runs[c] = runs;
    }
  });
  const int64_t first_bad = *std::min_element(bad.begin(), bad.end());
  if (first_bad != std::numeric_limits<int64_t>::max()) {
    std::snprintf(msg, sizeof msg, "voxel %lld has label %d > 1 + n_iolets", (long long)first_bad,
                  (int)labels[first_bad]);
    err = msg;
    return LBM_EINVAL;
  }
  std::vector<int64_t> col_base(C + 1), run_base(C + 1);
  col_base[0] = run_base[0] = 0;
  for (int64_t c = 0; c < C; ++c) {
    col_base[c + 1] = col_base[c] + col_n[c];
    run_base[c + 1] = run_base[c] + col_runs[c];
  }
  const int64_t n = col_base[C];
  // site ids are 32-bit, and so is the padded row length (n plus at most 191)
  if (n >= std::numeric_limits<int32_t>::max() - 8 * kTile) {
    err = "too many fluid sites for 32-bit site ids";
    return LBM_EINVAL;
  }
  col_n.clear();
  col_n.shrink_to_fit();
  col_runs.clear();
  col_runs.shrink_to_fit();
  struct Run {
    int32_t z0, z1, base;  // fluid voxels z0 <= z < z1 hold sites base + (z - z0)
  };
  std::vector<Run> runs(run_base[C]);
  L.nx = nx; L.ny = ny; L.nz = nz; L.n = n;
  L.coords.clear();
  L.coords.resize((size_t)3 * n);  // every element written below
  L.nbr.clear();
  L.nbr.resize((size_t)18 * n);
  parallel_for(C, [&](int64_t c0, int64_t c1, int) {
    for (int64_t c = c0; c < c1; ++c) {
      if (run_base[c + 1] == run_base[c]) continue;
      const uint8_t* lab = labels + c * nz;
      const int32_t x = (int32_t)(c / ny), y = (int32_t)(c % ny);
      int64_t s = col_base[c], r = run_base[c];
      bool in = false;
      for (int32_t z = 0; z < nz; ++z) {
        const bool f = lab[z] == 1;
        if (f && !in) runs[r] = Run{z, z, (int32_t)s};
        if (f) {
          runs[r].z1 = z + 1;
          int32_t* co = &L.coords[(size_t)3 * s];
          co[0] = x; co[1] = y; co[2] = z;
          ++s;
        } else if (in) {
          ++r;
        }
        in = f;
      }
    }
  });
  auto site_at = [&](int32_t X, int32_t Y, int32_t Z) -> int32_t {
    const int64_t c = (int64_t)X * ny + Y;
    for (int64_t r = run_base[c]; r < run_base[c + 1]; ++r)
      if (Z >= runs[r].z0 && Z < runs[r].z1) return runs[r].base + (Z - runs[r].z0);
    return -1;  // not reached for a voxel labelled fluid
  };
  // ---- links: site id, -1 wall, -2-k iolet k
  parallel_for(n, [&](int64_t s0, int64_t s1, int) {
    for (int64_t s = s0; s < s1; ++s) {
      const int32_t* co = &L.coords[(size_t)3 * s];
      for (int i = 1; i < kQ; ++i) {
        const int32_t X = co[0] + dir_x(i), Y = co[1] + dir_y(i), Z = co[2] + dir_z(i);
        int32_t code = -1;
        if (X >= 0 && Y >= 0 && Z >= 0 && X < nx && Y < ny && Z < nz) {
          const int lab = labels[((int64_t)X * ny + Y) * nz + Z];
          code = lab == 0 ? -1 : lab == 1 ? site_at(X, Y, Z) : -2 - (lab - 2);
        }
        L.nbr[(size_t)18 * s + (i - 1)] = code;
      }
    }
  });
  runs.clear();
  runs.shrink_to_fit();
  // ---- per-site summary: link masks, iolet links, the site's iolet id
  std::vector<uint32_t> site_mask(n, 0), site_io(n, 0);
  std::vector<int32_t> site_inlet(n, -1);
  std::vector<uint8_t> site_walls(n, 0);
  struct Clash {
    int64_t s;
    int a, b;
  };
  std::vector<Clash> clash(nthr, Clash{std::numeric_limits<int64_t>::max(), 0, 0});
  parallel_for(n, [&](int64_t s0, int64_t s1, int t) {
    for (int64_t s = s0; s < s1; ++s) {
      uint32_t m = 0, io = 0;
      int walls = 0, first_io = -1, inlet = -1;
      const int32_t* nb = &L.nbr[(size_t)18 * s];
      for (int i = 1; i < kQ; ++i) {
        const int32_t c = nb[i - 1];
        if (c >= 0) continue;
        m |= 1u << i;
        if (c == -1) {
          ++walls;
          m |= kHasWall;
          continue;
        }
        const int k = -2 - c;
        io |= 1u << i;
        if (first_io < 0) first_io = k;
        else if (first_io != k) m |= kMultiIolet;
        if (iolets[k].kind == LBM_IOLET_VELOCITY) {
          if (inlet >= 0 && inlet != k && clash[t].s == std::numeric_limits<int64_t>::max())
            clash[t] = Clash{s, inlet, k};
          inlet = k;
          m |= kHasInlet;
        }
      }
      const int id = inlet >= 0 ? inlet : first_io;
      if (id >= 0) io |= (uint32_t)id << kIoletShift;
      site_mask[s] = m;
      site_io[s] = io;
      site_inlet[s] = inlet;
      site_walls[s] = (uint8_t)walls;
    }
  });
  const Clash cl = *std::min_element(clash.begin(), clash.end(),
                                     [](const Clash& a, const Clash& b) { return a.s < b.s; });
  if (cl.s != std::numeric_limits<int64_t>::max()) {
    std::snprintf(msg, sizeof msg, "site %lld touches two velocity inlets (%d, %d)",
                  (long long)cl.s, cl.a, cl.b);
    err = msg;
    return LBM_EINVAL;
  }
  L.wall_sites.clear();
  L.n_wall_links = 0;
  std::vector<std::vector<int64_t>> io_sites(n_iolets);
  for (int64_t s = 0; s < n; ++s) {
    if (site_walls[s]) {
      L.wall_sites.push_back(s);
      L.n_wall_links += site_walls[s];
    }
    if (!(site_io[s] & kDirBits)) continue;
    const int32_t* nb = &L.nbr[(size_t)18 * s];
    for (int i = 1; i < kQ; ++i) {
      const int32_t c = nb[i - 1];
      if (c > -2) continue;
      const int k = -2 - c;
      if (io_sites[k].empty() || io_sites[k].back() != s) io_sites[k].push_back(s);
    }
  }
  site_walls.clear();
  site_walls.shrink_to_fit();
  L.iolet_off.assign(n_iolets + 1, 0);
  L.iolet_sites.clear();
  for (int k = 0; k < n_iolets; ++k) {
    L.iolet_sites.insert(L.iolet_sites.end(), io_sites[k].begin(), io_sites[k].end());
    L.iolet_off[k + 1] = (int64_t)L.iolet_sites.size();
  }
  // ---- tiles: classified in parallel, then numbered in order
  const int64_t T = (n + kTile - 1) / kTile;
  L.n_tiles = T;
  L.tiles.assign(T, TileDesc{});
  std::vector<uint8_t> tile_class(T, 0);  // 0 bulk, 1 coherent boundary, 2 irregular
  parallel_for(T, [&](int64_t t0, int64_t t1, int) {
    for (int64_t t = t0; t < t1; ++t) {
      const int64_t x0 = t * kTile;
      const int lanes = (int)std::min<int64_t>(kTile, n - x0);
      TileDesc& d = L.tiles[t];
      d.slot = -1;
      uint32_t flags = 0, nonfluid = 0;
      for (int l = 0; l < lanes; ++l) {
        flags |= site_mask[x0 + l] & (kHasWall | kHasInlet);
        nonfluid |= site_mask[x0 + l] & kDirBits;
      }
      // coherent: in every direction, the lanes whose link is fluid share one offset
      bool coherent = true;
      for (int i = 1; i < kQ && coherent; ++i) {
        bool have = false;
        int64_t off = 0;
        for (int l = 0; l < lanes; ++l) {
          const int32_t c = L.nbr[(size_t)18 * (x0 + l) + (i - 1)];
          if (c < 0) continue;
          const int64_t o = (int64_t)c - (x0 + l);
          if (!have) {
            have = true;
            off = o;
          } else if (o != off) {
            coherent = false;
            break;
          }
        }
        d.code[i - 1] = (int32_t)off;
      }
      if (coherent && nonfluid == 0) {
        tile_class[t] = 0;
        continue;
      }
      if (!coherent) {
        for (int i = 0; i < 18; ++i) d.code[i] = 0;
        d.mask = kIrregular;
        tile_class[t] = 2;
      } else {
        d.mask = nonfluid;
        tile_class[t] = 1;
      }
      d.mask |= flags;
    }
  });
  L.n_bulk = L.n_uniform = L.n_irregular = L.bulk_sites = 0;
  int64_t nb_tiles = 0;  // boundary tiles so far
  for (int64_t t = 0; t < T; ++t) {
    if (tile_class[t] == 0) {
      ++L.n_bulk;
      L.bulk_sites += std::min<int64_t>(kTile, n - t * kTile);
      continue;
    }
    if (tile_class[t] == 2) ++L.n_irregular;
    else ++L.n_uniform;
    L.tiles[t].slot = (int32_t)(nb_tiles * kTile);
    ++nb_tiles;
  }
  L.launch.clear();
  L.launch.reserve(T);
  for (int pass = 0; pass < 2; ++pass)
    for (int64_t t = 0; t < T; ++t) {
      const TileDesc& d = L.tiles[t];
      if ((d.slot >= 0) != (pass == 0)) continue;
      LaunchDesc e;
      for (int i = 0; i < 18; ++i) e.code[i] = d.code[i];
      e.mask = d.mask;
      e.tile = (int32_t)t;
      L.launch.push_back(e);
    }
  // ---- boundary slots
  const int64_t S = nb_tiles * kTile;
  L.n_slots = S;
  L.slot_mask.assign(S, 0);
  L.slot_io.assign(S, 0);
  L.slot_nbr.clear();
  L.slot_nbr.resize((size_t)18 * S);  // rows of boundary tiles written below; padding lanes zeroed
  parallel_for(S / kTile, [&](int64_t b0, int64_t b1, int) {
    for (int64_t b = b0; b < b1; ++b)
      for (int i = 0; i < 18; ++i)
        std::fill_n(&L.slot_nbr[(size_t)i * S + b * kTile], kTile, 0);
  });
  L.slot_prof.assign((size_t)3 * S, 0.0);
  const double nu = (tau - 0.5) / 3.0;  // Eq. (Viscosity), c_s^2 = 1/3
  std::vector<int64_t> slot_of(n, -1);
  parallel_for(T, [&](int64_t t0, int64_t t1, int) {
  for (int64_t t = t0; t < t1; ++t) {
    const TileDesc& d = L.tiles[t];
    if (d.slot < 0) continue;
    const int64_t x0 = t * kTile;
    const int lanes = (int)std::min<int64_t>(kTile, n - x0);
    for (int l = 0; l < lanes; ++l) {
      const int64_t x = x0 + l, m = (int64_t)d.slot + l;
      slot_of[x] = m;
      L.slot_mask[m] = site_mask[x] | kValid;
      L.slot_io[m] = site_io[x];
      for (int i = 0; i < 18; ++i) L.slot_nbr[(size_t)i * S + m] = L.nbr[(size_t)18 * x + i];
      const int k = site_inlet[x];
      if (k < 0) continue;
      const lbm_iolet& io = iolets[k];
      const double an = std::sqrt(io.axis[0] * io.axis[0] + io.axis[1] * io.axis[1] +
                                  io.axis[2] * io.axis[2]);
      double dd = 0.0, along = 0.0;
      for (int c = 0; c < 3; ++c) {
        const double dc = (double)L.coords[(size_t)3 * x + c] - io.centre[c];
        dd += dc * dc;
        along += dc * io.axis[c] / an;
      }
      double p0, ps, pc = 0.0;
      if (io.profile == LBM_PROFILE_PLUG) {
        p0 = ps = 1.0;
      } else {
        const double q = (dd - along * along) / (io.radius * io.radius);
        p0 = q < 1.0 ? 2.0 * (1.0 - q) : 0.0;
        ps = p0;
        if (io.profile == LBM_PROFILE_WOMERSLEY) {
          ps = 0.0;
          if (q < 1.0) {
            const double alpha =
                io.period > 0.0 ? io.radius * std::sqrt(2.0 * M_PI / io.period / nu) : 0.0;
            const cplx sh = womersley(alpha, std::sqrt(std::max(q, 0.0)));
            ps = sh.real();
            pc = sh.imag();
          }
        }
      }
      L.slot_prof[m] = p0;
      L.slot_prof[(size_t)S + m] = ps;
      L.slot_prof[(size_t)2 * S + m] = pc;
    }
  }
  });
  // segment tables of irregular tiles: split the lanes greedily into runs
  // that share one offset per direction (links leaving the fluid constrain
  // nothing); tiles that need at most kMaxSegments runs are marked kSegmented
  L.seg_tab.assign((size_t)nb_tiles * kSegWords, 0);
  parallel_for(T, [&](int64_t t0, int64_t t1, int) {
    for (int64_t t = t0; t < t1; ++t) {
      TileDesc& td = L.tiles[t];
      if (td.slot < 0 || !(td.mask & kIrregular)) continue;
      const int64_t x0 = t * kTile;
      const int lanes = (int)std::min<int64_t>(kTile, n - x0);
      int32_t* st = &L.seg_tab[(size_t)(td.slot / kTile) * kSegWords];
      int32_t off[18];
      bool have[18];
      int nseg = 0;
      bool ok = true;
      for (int l = 0; l < lanes && ok; ++l) {
        const int32_t* nb = &L.nbr[(size_t)18 * (x0 + l)];
        bool fits = nseg > 0;
        for (int i = 0; i < 18 && fits; ++i)
          if (nb[i] >= 0 && have[i] && nb[i] - (int32_t)(x0 + l) != off[i]) fits = false;
        if (!fits) {  // start a segment at lane l
          if (nseg == kMaxSegments) {
            ok = false;
            break;
          }
          st[nseg++] = l;
          for (int i = 0; i < 18; ++i) have[i] = false;
        }
        for (int i = 0; i < 18; ++i)
          if (nb[i] >= 0 && !have[i]) {
            have[i] = true;
            off[i] = nb[i] - (int32_t)(x0 + l);
          }
        for (int i = 0; i < 18; ++i) st[4 + 18 * (nseg - 1) + i] = have[i] ? off[i] : 0;
      }
      if (!ok) {
        std::fill(st, st + kSegWords, 0);
        continue;
      }
      for (int q = nseg; q < kMaxSegments; ++q) st[q] = kTile;
      td.mask |= kSegmented;
    }
  });
  for (LaunchDesc& e : L.launch)
    if (e.mask & kIrregular) e.mask = L.tiles[e.tile].mask;
  L.multi_tiles.clear();
  for (int64_t b = 0; b < nb_tiles; ++b)
    for (int l = 0; l < kTile; ++l)
      if (L.slot_mask[b * kTile + l] & kMultiIolet) {
        L.multi_tiles.push_back((int32_t)b);  // boundary tiles lead the launch order
        break;
      }
  L.wall_slot.resize(L.wall_sites.size());
  parallel_for((int64_t)L.wall_sites.size(), [&](int64_t w0, int64_t w1, int) {
    for (int64_t w = w0; w < w1; ++w) L.wall_slot[w] = slot_of[L.wall_sites[w]];
  });
  return LBM_OK;
}

}  // namespace lbm

// --------------------------------------------------------------- F map
// Host precompute of F (Sec. 2.3, Eq. F) over a grid of (alpha, dr/R).

extern "C" int lbm_fmap(const double* alpha, int64_t n_alpha, const double* dr_over_R,
                        int64_t n_dr, double M_re, double M_im, double* out) {
  using lbm::cplx;
  if (n_alpha < 0 || n_dr < 0 || ((n_alpha > 0 && n_dr > 0) && (!alpha || !dr_over_R || !out)) ||
      !std::isfinite(M_re) || !std::isfinite(M_im))
    return LBM_EINVAL;
  for (int64_t a = 0; a < n_alpha; ++a)
    if (!(alpha[a] >= 0.0 && alpha[a] <= 25.0)) return LBM_EINVAL;
  for (int64_t b = 0; b < n_dr; ++b)
    if (!(dr_over_R[b] >= 0.0 && dr_over_R[b] < 1.0)) return LBM_EINVAL;
  const cplx M(M_re, M_im);
  for (int64_t a = 0; a < n_alpha; ++a) {
    const cplx lam = alpha[a] * std::exp(cplx(0.0, 0.75 * M_PI));
    cplx j0L, j1L;
    lbm::bessel01(lam, j0L, j1L);
    for (int64_t b = 0; b < n_dr; ++b) {
      cplx j0r, j1r;
      lbm::bessel01(lam * (1.0 - dr_over_R[b]), j0r, j1r);
      const cplx den = 1.0 - M * j0r / j0L;
      cplx F;
      if (std::abs(den) == 0.0) F = cplx(NAN, NAN);
      else F = (1.0 - M) / den;
      out[2 * (a * n_dr + b)] = F.real();
      out[2 * (a * n_dr + b) + 1] = F.imag();
    }
  }
  return LBM_OK;
}
