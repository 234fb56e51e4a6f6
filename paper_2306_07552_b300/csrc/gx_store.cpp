// Box store of a scene's static distance field (host build).  The distance
// grid is the signed distance of the union of the scene's solid boxes,
// sampled at lattice nodes (appendix "Additional Collision-Detection
// Details" precomputes the static structure; here it is a lattice of signed
// distances).  Instead of storing every node, the box store keeps the boxes
// and, per cell of 16 node intervals per axis, the boxes that can be the
// nearest one somewhere in the cell; the kernels recompute a node as the
// minimum over that short list.
//
// Candidate test, in FP64: the signed distance sd_b of a box is convex, so
// over an axis-aligned region R its maximum U_b is reached at a corner of R;
// a lower bound L_b of its minimum is the distance between R and the box
// when they are disjoint, else the largest per-axis lower bound of the
// inside term.  At any point of R the field is at most U* = min_b U_b, and
// box b exceeds it everywhere when L_b > U*, so the boxes with L_b <= U*
// contain the argmin of every point of R.  R is widened by 0.1 mm so that
// the kernels' FP32 node positions and FP32 box copies stay inside it.
#include <algorithm>
#include <cmath>

#include "gx_internal.h"

namespace gx {

namespace {

double box_sd(const double p[3], const double c[3], const double e[3]) {
  double out2 = 0.0, inmax = -1e300;
  for (int a = 0; a < 3; ++a) {
    const double q = std::fabs(p[a] - c[a]) - e[a];
    out2 += q > 0.0 ? q * q : 0.0;
    inmax = std::max(inmax, q);
  }
  return std::sqrt(out2) + std::min(inmax, 0.0);
}

}  // namespace

bool build_box_store(const gx_scene_desc& d, StoreHost& out) {
  const int nx = d.grid_dims[0], ny = d.grid_dims[1], nz = d.grid_dims[2];
  const int C = 1 << kStoreShift;
  out.sbx = std::max(1, (nx - 1 + C - 1) / C);
  out.sby = std::max(1, (ny - 1 + C - 1) / C);
  out.sbz = std::max(1, (nz - 1 + C - 1) / C);
  const int nb = d.n_boxes;
  std::vector<double> bc(3 * (size_t)nb), be(3 * (size_t)nb);
  out.boxes.resize(2 * (size_t)nb);
  for (int b = 0; b < nb; ++b) {
    double c[3], e[3];
    for (int a = 0; a < 3; ++a) {
      const double lo = d.boxes[6 * b + a], hi = d.boxes[6 * b + 3 + a];
      c[a] = 0.5 * (lo + hi);
      e[a] = 0.5 * (hi - lo);
      bc[3 * b + a] = c[a];
      be[3 * b + a] = e[a];
    }
    out.boxes[2 * b] = make_float4((float)c[0], (float)c[1], (float)c[2], 0.f);
    out.boxes[2 * b + 1] = make_float4((float)e[0], (float)e[1], (float)e[2], 0.f);
  }
  const double h = d.grid_h, o[3] = {d.grid_origin[0], d.grid_origin[1], d.grid_origin[2]};
  const int n[3] = {nx, ny, nz};
  const size_t cells = (size_t)out.sbx * out.sby * out.sbz;
  out.off.assign(cells + 1, 0);
  out.ids.clear();
  std::vector<double> L(nb), U(nb);
  for (int ck = 0; ck < out.sbz; ++ck)
    for (int cj = 0; cj < out.sby; ++cj)
      for (int ci = 0; ci < out.sbx; ++ci) {
        const int cidx[3] = {ci, cj, ck};
        double rlo[3], rhi[3];
        for (int a = 0; a < 3; ++a) {
          const int i0 = cidx[a] * C, i1 = std::min(cidx[a] * C + C, n[a] - 1);
          rlo[a] = o[a] + i0 * h - 1e-4;
          rhi[a] = o[a] + i1 * h + 1e-4;
        }
        double ustar = 1e300;
        for (int b = 0; b < nb; ++b) {
          const double* c = &bc[3 * b];
          const double* e = &be[3 * b];
          double u = -1e300;
          for (int v = 0; v < 8; ++v) {
            const double p[3] = {(v & 1) ? rhi[0] : rlo[0], (v & 2) ? rhi[1] : rlo[1],
                                 (v & 4) ? rhi[2] : rlo[2]};
            u = std::max(u, box_sd(p, c, e));
          }
          U[b] = u;
          ustar = std::min(ustar, u);
          double gap2 = 0.0, inl = -1e300;
          bool apart = false;
          for (int a = 0; a < 3; ++a) {
            const double blo = c[a] - e[a], bhi = c[a] + e[a];
            const double g = std::max(0.0, std::max(blo - rhi[a], rlo[a] - bhi));
            if (g > 0.0) apart = true;
            gap2 += g * g;
            const double m = (c[a] >= rlo[a] && c[a] <= rhi[a])
                                 ? 0.0
                                 : std::min(std::fabs(rlo[a] - c[a]), std::fabs(rhi[a] - c[a]));
            inl = std::max(inl, m - e[a]);
          }
          L[b] = apart ? std::sqrt(gap2) : inl;
        }
        const size_t cell = ((size_t)ck * out.sby + cj) * out.sbx + ci;
        for (int b = 0; b < nb; ++b)
          if (L[b] <= ustar + 1e-9) out.ids.push_back((uint16_t)b);
        out.off[cell + 1] = (uint32_t)out.ids.size();
        if (out.ids.size() >= ((size_t)1 << 32)) return false;
      }
  return true;
}

}  // namespace gx

// Host-only view of the candidate lists (the same build gx_scene_set_create
// uploads); touches no device.
extern "C" gx_status gx_box_store_lists(const gx_scene_desc* scene, int32_t dims[3],
                                        uint32_t* offsets, uint16_t* ids, uint64_t* n_ids) {
  if (!scene || !dims || !n_ids || scene->n_boxes < 1 || scene->n_boxes > 4096 ||
      !scene->boxes || !(scene->grid_h > 0.f) || scene->grid_dims[0] < 2 ||
      scene->grid_dims[1] < 2 || scene->grid_dims[2] < 2)
    return gx::set_last_error(GX_EINVAL, "gx_box_store_lists: bad scene");
  gx::StoreHost sh;
  if (!gx::build_box_store(*scene, sh))
    return gx::set_last_error(GX_EINVAL, "gx_box_store_lists: box store too large");
  dims[0] = sh.sbx;
  dims[1] = sh.sby;
  dims[2] = sh.sbz;
  *n_ids = sh.ids.size();
  if (offsets) std::copy(sh.off.begin(), sh.off.end(), offsets);
  if (ids) std::copy(sh.ids.begin(), sh.ids.end(), ids);
  return GX_OK;
}
