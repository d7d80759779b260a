// Tile planner of the fused branch-A sweep step (host; kernel in
// sweep_fused.cu).
//
// A grid (lx, lv) is cut into x patches (vertex sets of level lx of Omega_x)
// and v patches (vertex sets of level lv of Omega_v) by recursive coordinate
// bisection: split along the longest extent at the median until a patch has
// at most B vertices, which keeps patches compact on any mesh and in any
// dimension.  A tile pairs one x patch with one v patch.
//  - Its rows: the x patch (interior) and the vertices the level pattern
//    reaches from it (halo): the X stencils of the interior outputs read S_b
//    there.
//  - Its columns: the v patch (interior) and, when the grid passes states on
//    (i < L), the fine vertices reached by the restriction rows of the coarse
//    vertices the patch owns (a coarse vertex belongs to the patch holding
//    its injected fine vertex).
// The patch sizes are chosen per grid from a few candidates by a cost model:
// S_b entries formed (interior and halo) x chains, plus one U gather per
// entry and chain group, plus the final update per output and term, plus a
// fixed cost per tile and chain group; subject to the tile's S_b fitting in
// shared memory for at least one chain and its interior fitting the block's
// output registers.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "handle.h"

namespace sgdg {

namespace {

constexpr size_t kFusedSmem = 220 * 1024;   // dynamic shared memory per block (1 block per SM)

struct Patches {
  std::vector<int> ids;                    // vertices, patch by patch (interior sorted, then halo sorted)
  std::vector<int> beg, nint, ntot;        // per patch: offset into ids, interior and total counts
  std::vector<int> qbeg, nq;               // v side: owned coarse vertices (qcols offsets)
  std::vector<int> qcols;
  std::vector<unsigned short> loc;         // x: [interior][W] local rows; v: [owned][W] local columns
  std::vector<int> locbeg;                 // per patch: offset into loc
  long long sum_tot = 0, sum_q = 0;
  int max_int = 0, max_tot = 0, count = 0;
  bool ok = true;
};

void rcb(const std::vector<double>& coords, int d, std::vector<int>& ids, int lo, int hi, int B,
         std::vector<std::pair<int, int>>& parts) {
  if (hi - lo <= B) {
    parts.push_back({lo, hi});
    return;
  }
  int axis = 0;
  double best = -1.0;
  for (int k = 0; k < d; ++k) {
    double mn = 1e300, mx = -1e300;
    for (int p = lo; p < hi; ++p) {
      const double x = coords[(size_t)ids[p] * d + k];
      mn = std::min(mn, x);
      mx = std::max(mx, x);
    }
    if (mx - mn > best) { best = mx - mn; axis = k; }
  }
  const int mid = lo + (hi - lo) / 2;
  std::nth_element(ids.begin() + lo, ids.begin() + mid, ids.begin() + hi, [&](int a, int b) {
    const double xa = coords[(size_t)a * d + axis], xb = coords[(size_t)b * d + axis];
    return xa < xb || (xa == xb && a < b);
  });
  rcb(coords, d, ids, lo, mid, B, parts);
  rcb(coords, d, ids, mid, hi, B, parts);
}

// x side: patches of level-lx vertices; halo = pattern neighbours of the
// interior; loc[r][j] = local row of ELL entry j of interior row r.
Patches x_patches(const MeshLevel& lev, int d, const std::vector<int>& ell, int W, int B) {
  Patches P;
  const int n = lev.n;
  std::vector<int> ids(n);
  std::iota(ids.begin(), ids.end(), 0);
  std::vector<std::pair<int, int>> parts;
  rcb(lev.coords, d, ids, 0, n, B, parts);
  std::vector<int> stamp(n, -1), local(n, -1);
  for (size_t pi = 0; pi < parts.size(); ++pi) {
    std::vector<int> in(ids.begin() + parts[pi].first, ids.begin() + parts[pi].second);
    std::sort(in.begin(), in.end());
    for (int k : in) stamp[k] = (int)pi;
    std::vector<int> halo;
    for (int k : in)
      for (int j = 0; j < W; ++j) {
        const int c = ell[(size_t)k * W + j];
        if (stamp[c] != (int)pi) {
          stamp[c] = (int)pi;
          halo.push_back(c);
        }
      }
    std::sort(halo.begin(), halo.end());
    P.beg.push_back((int)P.ids.size());
    P.nint.push_back((int)in.size());
    P.ntot.push_back((int)(in.size() + halo.size()));
    int r = 0;
    for (int k : in) local[k] = r++;
    for (int k : halo) local[k] = r++;
    P.ids.insert(P.ids.end(), in.begin(), in.end());
    P.ids.insert(P.ids.end(), halo.begin(), halo.end());
    P.locbeg.push_back((int)P.loc.size());
    if (r > 65535) P.ok = false;
    for (int k : in)
      for (int j = 0; j < W; ++j) P.loc.push_back((unsigned short)local[ell[(size_t)k * W + j]]);
    P.sum_tot += r;
    P.max_int = std::max(P.max_int, (int)in.size());
    P.max_tot = std::max(P.max_tot, r);
  }
  P.count = (int)parts.size();
  return P;
}

// v side: patches of level-lv vertices; with restriction (R: level lv-1 rows,
// ELL width W; inj: level lv-1 vertex -> level lv index) every coarse vertex
// belongs to the patch holding its injected vertex, and the halo holds the
// fine vertices its restriction row reaches.
Patches v_patches(const MeshLevel& lev, int d, const std::vector<int>* rell, const std::vector<int>* inj, int W,
                  int B) {
  Patches P;
  const int n = lev.n;
  std::vector<int> ids(n);
  std::iota(ids.begin(), ids.end(), 0);
  std::vector<std::pair<int, int>> parts;
  rcb(lev.coords, d, ids, 0, n, B, parts);
  std::vector<int> owner(n, -1), stamp(n, -1), local(n, -1);
  for (size_t pi = 0; pi < parts.size(); ++pi)
    for (int p = parts[pi].first; p < parts[pi].second; ++p) owner[ids[p]] = (int)pi;
  std::vector<std::vector<int>> owned(parts.size());
  if (rell)
    for (int c = 0; c < (int)inj->size(); ++c) owned[owner[(*inj)[c]]].push_back(c);
  for (size_t pi = 0; pi < parts.size(); ++pi) {
    std::vector<int> in(ids.begin() + parts[pi].first, ids.begin() + parts[pi].second);
    std::sort(in.begin(), in.end());
    for (int k : in) stamp[k] = (int)pi;
    std::vector<int> halo;
    for (int c : owned[pi])
      for (int j = 0; j < W; ++j) {
        const int f = (*rell)[(size_t)c * W + j];
        if (stamp[f] != (int)pi) {
          stamp[f] = (int)pi;
          halo.push_back(f);
        }
      }
    std::sort(halo.begin(), halo.end());
    P.beg.push_back((int)P.ids.size());
    P.nint.push_back((int)in.size());
    P.ntot.push_back((int)(in.size() + halo.size()));
    int r = 0;
    for (int k : in) local[k] = r++;
    for (int k : halo) local[k] = r++;
    P.ids.insert(P.ids.end(), in.begin(), in.end());
    P.ids.insert(P.ids.end(), halo.begin(), halo.end());
    P.qbeg.push_back((int)P.qcols.size());
    P.nq.push_back((int)owned[pi].size());
    P.qcols.insert(P.qcols.end(), owned[pi].begin(), owned[pi].end());
    for (int c : owned[pi])
      for (int j = 0; j < W; ++j) P.loc.push_back((unsigned short)local[(*rell)[(size_t)c * W + j]]);
    if (r > 65535) P.ok = false;
    P.sum_tot += r;
    P.sum_q += (long long)owned[pi].size();
    P.max_int = std::max(P.max_int, (int)in.size());
    P.max_tot = std::max(P.max_tot, r);
  }
  P.count = (int)parts.size();
  return P;
}

std::vector<int> candidates(int n) {
  std::vector<int> c;
  for (int b : {16, 32, 64, 128, 256, 512, 1024, 2048, 4096})
    if (b < n) c.push_back(b);
  c.push_back(n);
  return c;
}

template <typename T>
Status upload_vec(Handle& h, T** dst, const std::vector<T>& v) {
  if (dev_alloc(h, (void**)dst, sizeof(T) * std::max<size_t>(v.size(), 1)) != cudaSuccess)
    return {SGDG_ENOMEM, "fused sweep plan"};
  if (!v.empty() && cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return {SGDG_ECUDA, "fused sweep plan upload"};
  return {};
}

}  // namespace

Status fused_plan(Handle& h, int i, int pair_bytes, int nchains, int nterms, const Handle::FusedGrid** out) {
  *out = nullptr;
  const long long key = (long long)i * 64 + pair_bytes;
  Handle::FusedGrid& fg = h.fused[key];
  if (fg.tried) {
    if (fg.ok && fg.G > 0) *out = &fg;
    return {};
  }
  fg.tried = true;
  if (!h.hx_host || !h.hv_host) { fg.why = "no host hierarchy"; return {}; }
  if (nchains < 1 || nchains > kFusedChains || nterms > kFusedTerms) { fg.why = "too many chains or terms"; return {}; }
  const int W = h.X.ell_w();
  if (h.V.ell_w() != W || (W != 4 && W != 8 && W != 16)) { fg.why = "ELL widths differ"; return {}; }
  const int L = h.L, lx = i, lv = L - i;
  const Hierarchy& HX = *h.hx_host;
  const Hierarchy& HV = *h.hv_host;
  const MeshLevel& xl = HX.lev[lx];
  const MeshLevel& vl = HV.lev[lv];
  const std::vector<int> xell = pattern_ell_columns(h.X, xl.pattern, lx);
  const bool restrict_out = i < L;
  std::vector<int> rell;
  if (restrict_out) rell = ell_columns(HV.Rt[lv - 1].rowptr, HV.Rt[lv - 1].col, W);
  const std::vector<int>* inj = restrict_out ? &HV.inj[lv - 1] : nullptr;
  // candidate patchings per side
  std::vector<Patches> xs, vs;
  for (int b : candidates(xl.n)) {
    xs.push_back(x_patches(xl, HX.d, xell, W, b));
    if (xl.n <= 4096 && b < xl.n && xs.back().max_tot >= xl.n) xs.pop_back();   // no gain over all rows
  }
  for (int b : candidates(vl.n)) vs.push_back(v_patches(vl, HV.d, restrict_out ? &rell : nullptr, inj, W, b));
  const double n_out = (double)xl.n * vl.n;
  double best = 1e300;
  int bx = -1, bv = -1, bG = 0;
  for (size_t a = 0; a < xs.size(); ++a) {
    for (size_t b = 0; b < vs.size(); ++b) {
      const Patches& X = xs[a];
      const Patches& V = vs[b];
      if (!X.ok || !V.ok) continue;
      if ((long long)X.max_int * V.max_int > (long long)kFusedThreads * kFusedOut) continue;
      const size_t per_chain = (size_t)X.max_tot * V.max_tot * pair_bytes;
      if (per_chain > kFusedSmem) continue;
      int G = (int)std::min<size_t>(nchains, kFusedSmem / per_chain);
      const int ngroups = (nchains + G - 1) / G;
      G = (nchains + ngroups - 1) / ngroups;
      const double spts = (double)X.sum_tot * (double)V.sum_tot;
      const double tiles = (double)X.count * V.count;
      const double cost = spts * (nchains * 25.0 + ngroups * (W + 4.0)) + n_out * nterms * 27.0 +
                          (double)X.sum_tot * (double)V.sum_q * 0 + tiles * ngroups * 4000.0;
      if (cost < best) {
        best = cost;
        bx = (int)a;
        bv = (int)b;
        bG = G;
      }
    }
  }
  if (bx < 0) { fg.why = "no tile shape fits shared memory"; return {}; }
  const Patches& X = xs[bx];
  const Patches& V = vs[bv];
  std::vector<FusedTile> tiles;
  tiles.reserve((size_t)X.count * V.count);
  for (int a = 0; a < X.count; ++a)
    for (int b = 0; b < V.count; ++b) {
      FusedTile t;
      t.xs0 = X.beg[a];
      t.nxi = X.nint[a];
      t.nxt = X.ntot[a];
      t.xn0 = X.locbeg[a];
      t.vs0 = V.beg[b];
      t.nvi = V.nint[b];
      t.nvt = V.ntot[b];
      t.q0 = V.qbeg[b];
      t.nq = V.nq[b];
      tiles.push_back(t);
    }
  Status st = upload_vec(h, &fg.tiles, tiles);
  if (!st.code) st = upload_vec(h, &fg.xrows, X.ids);
  if (!st.code) st = upload_vec(h, &fg.vcols, V.ids);
  if (!st.code) st = upload_vec(h, &fg.xnbr, X.loc);
  if (!st.code) st = upload_vec(h, &fg.qcols, V.qcols);
  if (!st.code) st = upload_vec(h, &fg.qloc, V.loc);
  if (st.code) return st;
  fg.G = bG;
  fg.W = W;
  fg.ntiles = (int)tiles.size();
  fg.smem = (size_t)X.max_tot * V.max_tot * pair_bytes * bG;
  fg.s_points = (double)X.sum_tot * (double)V.sum_tot;
  fg.q_points = (double)xl.n * (double)V.sum_q;
  fg.ok = true;
  *out = &fg;
  return {};
}

}  // namespace sgdg
