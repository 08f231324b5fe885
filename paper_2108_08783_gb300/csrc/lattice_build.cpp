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
  const int64_t nvox = (int64_t)nx * ny * nz;
  const int max_label = 1 + n_iolets;
  std::vector<int32_t> site_of(nvox, -1);
  int64_t n = 0;
  for (int64_t v = 0; v < nvox; ++v) {
    if (labels[v] > max_label) {
      std::snprintf(msg, sizeof msg, "voxel %lld has label %d > 1 + n_iolets", (long long)v,
                    (int)labels[v]);
      err = msg;
      return LBM_EINVAL;
    }
    if (labels[v] == 1) {
      if (n >= std::numeric_limits<int32_t>::max() - 4 * kTile) {
        err = "too many fluid sites for 32-bit site ids";
        return LBM_EINVAL;
      }
      site_of[v] = (int32_t)n++;
    }
  }
  L.nx = nx; L.ny = ny; L.nz = nz; L.n = n;
  L.coords.assign((size_t)3 * n, 0);
  L.nbr.assign((size_t)18 * n, 0);
  // ---- links: site id, -1 wall, -2-k iolet k
  for (int32_t x = 0; x < nx; ++x)
    for (int32_t y = 0; y < ny; ++y)
      for (int32_t z = 0; z < nz; ++z) {
        const int64_t v = ((int64_t)x * ny + y) * nz + z;
        const int32_t s = site_of[v];
        if (s < 0) continue;
        int32_t* c = &L.coords[(size_t)3 * s];
        c[0] = x; c[1] = y; c[2] = z;
        for (int i = 1; i < kQ; ++i) {
          const int32_t X = x + dir_x(i), Y = y + dir_y(i), Z = z + dir_z(i);
          int32_t code = -1;
          if (X >= 0 && Y >= 0 && Z >= 0 && X < nx && Y < ny && Z < nz) {
            const int64_t w = ((int64_t)X * ny + Y) * nz + Z;
            const int lab = labels[w];
            code = lab == 0 ? -1 : lab == 1 ? site_of[w] : -2 - (lab - 2);
          }
          L.nbr[(size_t)18 * s + (i - 1)] = code;
        }
      }
  site_of.clear();
  site_of.shrink_to_fit();
  // ---- per-site summary: link masks, iolet links, the site's iolet id
  std::vector<uint32_t> site_mask(n, 0), site_io(n, 0);
  std::vector<int32_t> site_inlet(n, -1);
  L.wall_sites.clear();
  L.n_wall_links = 0;
  std::vector<std::vector<int64_t>> io_sites(n_iolets);
  for (int64_t s = 0; s < n; ++s) {
    uint32_t m = 0, io = 0;
    int walls = 0, first_io = -1;
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
      if (io_sites[k].empty() || io_sites[k].back() != s) io_sites[k].push_back(s);
      if (iolets[k].kind == LBM_IOLET_VELOCITY) {
        if (site_inlet[s] >= 0 && site_inlet[s] != k) {
          std::snprintf(msg, sizeof msg, "site %lld touches two velocity inlets (%d, %d)",
                        (long long)s, site_inlet[s], k);
          err = msg;
          return LBM_EINVAL;
        }
        site_inlet[s] = k;
        m |= kHasInlet;
      }
    }
    const int id = site_inlet[s] >= 0 ? site_inlet[s] : first_io;
    if (id >= 0) io |= (uint32_t)id << kIoletShift;
    site_mask[s] = m;
    site_io[s] = io;
    if (walls) L.wall_sites.push_back(s);
    L.n_wall_links += walls;
  }
  L.iolet_off.assign(n_iolets + 1, 0);
  L.iolet_sites.clear();
  for (int k = 0; k < n_iolets; ++k) {
    L.iolet_sites.insert(L.iolet_sites.end(), io_sites[k].begin(), io_sites[k].end());
    L.iolet_off[k + 1] = (int64_t)L.iolet_sites.size();
  }
  // ---- tiles
  const int64_t T = (n + kTile - 1) / kTile;
  L.n_tiles = T;
  L.tiles.assign(T, TileDesc{});
  L.n_bulk = L.n_uniform = L.n_irregular = L.bulk_sites = 0;
  int64_t nb_tiles = 0;  // boundary tiles so far
  for (int64_t t = 0; t < T; ++t) {
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
      ++L.n_bulk;
      L.bulk_sites += lanes;
      continue;
    }
    if (!coherent) {
      for (int i = 0; i < 18; ++i) d.code[i] = 0;
      d.mask = kIrregular;
      ++L.n_irregular;
    } else {
      d.mask = nonfluid;
      ++L.n_uniform;
    }
    d.mask |= flags;
    d.slot = (int32_t)(nb_tiles * kTile);
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
  L.slot_nbr.assign((size_t)18 * S, 0);
  L.slot_prof.assign((size_t)3 * S, 0.0);
  const double nu = (tau - 0.5) / 3.0;  // Eq. (Viscosity), c_s^2 = 1/3
  std::vector<int64_t> slot_of(n, -1);
  for (int64_t t = 0; t < T; ++t) {
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
  L.wall_slot.resize(L.wall_sites.size());
  for (size_t w = 0; w < L.wall_sites.size(); ++w) L.wall_slot[w] = slot_of[L.wall_sites[w]];
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
