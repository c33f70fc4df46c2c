// C ABI: setup (host assembly, subdomains, symbolic; device factorisation)
// and the flexible GMRES solve driven by the device kernels.
//
// Sec. "Domain decomposition preconditioner": GMRES on A u = b with the
// two-level preconditioner of Eq. 2lvl; the coarse problem solved by a fixed
// number of GMRES iterations preconditioned by one-level ORAS on the coarse
// mesh. GMRES is run right-preconditioned and flexible (the inner coarse
// iteration makes M^{-1} vary between applications), one Krylov space per
// right-hand side, so the monitored residual is the paper's
// ||A u - b|| / ||b|| (Sec. "Tetrahedral finite element method").
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <numeric>
#include <string>

#include "../../include/hz.h"
#include "dd_host.h"
#include "kernels.cuh"

namespace hz {
// harmonic Ritz vectors of an FGMRES cycle (ritz_host.cpp)
bool harmonic_ritz(const std::vector<std::complex<double>>& Hbar, int m, int k,
                   std::vector<std::complex<double>>& P, std::vector<std::complex<double>>& theta);
}  // namespace hz

using namespace hz;

namespace {

thread_local std::string g_last_error;

struct CudaFail {
  cudaError_t e;
  const char* what;
};

#define CK(x)                                     \
  do {                                            \
    cudaError_t _e = (x);                         \
    if (_e != cudaSuccess) throw CudaFail{_e, #x}; \
  } while (0)

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Device allocation tracker: every buffer of a context is released in hz_free.
struct DevPool {
  std::vector<void*> ptrs;
  double bytes = 0;
  template <typename T>
  T* alloc(size_t count) {
    if (count == 0) count = 1;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw HzError{HZ_ENOMEM, "device allocation of " + std::to_string(count * sizeof(T)) + " bytes failed"};
    }
    ptrs.push_back(p);
    bytes += count * sizeof(T);
    return (T*)p;
  }
  template <typename T>
  T* upload(const std::vector<T>& v, cudaStream_t st) {
    T* p = alloc<T>(v.size());
    if (!v.empty()) CK(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    return p;
  }
  void free_one(void* p, size_t nbytes) {
    auto it = std::find(ptrs.begin(), ptrs.end(), p);
    if (it == ptrs.end()) return;
    cudaFree(p);
    ptrs.erase(it);
    bytes -= nbytes;
  }
  void release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
    bytes = 0;
  }
};

struct MFHost {
  int64_t factor_entries = 0, front_entries = 0, stored_entries = 0;
  std::vector<int> fa_small_ptr, fa_big_ptr, fa_step_ptr, fa_tile_ptr, fi_tile_ptr;  // factorisation schedule
  int max_front = 0, nfronts = 0, nlevels = 0;
  std::vector<int> level_ptr, ftile_ptr, btile_ptr, frb_ptr, brb_ptr;
  std::vector<int> fs_ptr, bs_ptr, ftc_ptr, btc_ptr;  // tensor-core mode split of the tile lists
  std::vector<int64_t> level_row;
  // per-level algorithmic work of one solve sweep (complex multiply-adds per column)
  std::vector<double> fwd_cmacs, bwd_cmacs;
  // per level: every tile has at most 64 output rows (half-height tiles in the solve)
  std::vector<char> fhalf, bhalf;
};

// Pack the fronts of several local matrices into one device structure;
// sub_off[i] is the first row of subdomain i in the flat sub-vector.
constexpr int MF_TILE_ROWS = 128;  // output rows per sweep tile (MF_TILE in mf.cu)
constexpr int MF_TILE_K = 128;     // reduction length per sweep tile (MF_TK in mf.cu)

void build_mf(const std::vector<const CsrC*>& mats, const std::vector<const FrontTree*>& trees,
              const std::vector<int64_t>& sub_off, bool fp32, bool fr32, bool tc, bool persistent, DevMF& mf,
              MFHost& info, DevPool& pool, cudaStream_t st) {
  tc = tc && fp32;
  const size_t ns = mats.size();
  std::vector<int> base(ns + 1, 0);
  for (size_t i = 0; i < ns; ++i) base[i + 1] = base[i] + (int)trees[i]->k.size();
  const int nf = base[ns];
  std::vector<int> k(nf), f(nf), height(nf), child_ptr(nf + 1, 0), child_idx, parent(nf, -1);
  std::vector<int64_t> Foff(nf + 1, 0), rowoff(nf + 1, 0), Moff(nf + 1, 0), Doff(nf + 1, 0);
  for (size_t i = 0; i < ns; ++i) {
    const FrontTree& T = *trees[i];
    for (size_t t = 0; t < T.k.size(); ++t) {
      int g = base[i] + (int)t;
      k[g] = T.k[t];
      f[g] = T.k[t] + T.m[t];
      height[g] = T.height[t];
      parent[g] = T.parent[t] >= 0 ? base[i] + T.parent[t] : -1;
      info.factor_entries += (int64_t)T.k[t] * (T.k[t] + 1) / 2 + (int64_t)T.k[t] * T.m[t];
    }
  }
  // level schedule by tree height; front rows are laid out level by level so
  // that every level's rows form one contiguous range
  int maxh = 0;
  for (int g = 0; g < nf; ++g) maxh = std::max(maxh, height[g]);
  info.nlevels = maxh + 1;
  info.nfronts = nf;
  info.level_ptr.assign(maxh + 2, 0);
  for (int g = 0; g < nf; ++g) info.level_ptr[height[g] + 1]++;
  for (int l = 0; l <= maxh; ++l) info.level_ptr[l + 1] += info.level_ptr[l];
  std::vector<int> level_list(nf);
  {
    std::vector<int> fill(info.level_ptr.begin(), info.level_ptr.end() - 1);
    for (int g = 0; g < nf; ++g) level_list[fill[height[g]]++] = g;
  }
  {
    int64_t acc = 0;
    for (int q = 0; q < nf; ++q) {
      rowoff[level_list[q]] = acc;
      acc += f[level_list[q]];
    }
    rowoff[nf] = acc;
  }
  for (int g = 0; g < nf; ++g) {
    Foff[g + 1] = Foff[g] + (int64_t)f[g] * f[g];
    Moff[g + 1] = Moff[g] + (int64_t)f[g] * k[g];
    Doff[g + 1] = Doff[g] + k[g];
    info.max_front = std::max(info.max_front, f[g]);
    if ((int64_t)f[g] * f[g] >= (int64_t)1 << 31) throw HzError{HZ_EINVAL, "front too large"};
  }
  info.front_entries = Foff[nf];
  info.stored_entries = Moff[nf];
  std::vector<int> rows(rowoff[nf]), cmap(rowoff[nf], -1);
  std::vector<int64_t> amap_ptr(nf + 1, 0);
  std::vector<int> amap_pos;
  std::vector<int64_t> amap_val;
  std::vector<double2> Aval;
  for (size_t i = 0; i < ns; ++i) {
    const FrontTree& T = *trees[i];
    const CsrC& A = *mats[i];
    const int64_t aoff = (int64_t)Aval.size();
    for (const cplx& v : A.val) Aval.push_back(make_double2(v.real(), v.imag()));
    const int ntf = (int)T.k.size();
    // front position of a local row v inside front t
    auto front_pos = [&](int t, int32_t v) -> int {
      int p = T.pos[v];
      if (p >= T.piv_begin[t] && p < T.piv_begin[t] + T.k[t]) return (int)(p - T.piv_begin[t]);
      const int32_t* ub = &T.upd[T.upd_ptr[t]];
      int lo = 0, hi = T.m[t];
      while (lo < hi) {  // update rows are sorted by elimination position
        int mid = (lo + hi) / 2;
        if (T.pos[ub[mid]] < p)
          lo = mid + 1;
        else
          hi = mid;
      }
      if (lo >= T.m[t] || ub[lo] != v) return -1;
      return T.k[t] + lo;
    };
    for (int t = 0; t < ntf; ++t) {
      const int g = base[i] + t;
      int64_t ro = rowoff[g];
      for (int r = 0; r < T.k[t]; ++r) rows[ro + r] = (int)(sub_off[i] + T.perm[T.piv_begin[t] + r]);
      for (int q = 0; q < T.m[t]; ++q) rows[ro + T.k[t] + q] = (int)(sub_off[i] + T.upd[T.upd_ptr[t] + q]);
      if (T.parent[t] >= 0)
        for (int q = 0; q < T.m[t]; ++q) {
          int pp = front_pos(T.parent[t], T.upd[T.upd_ptr[t] + q]);
          if (pp < 0) throw HzError{HZ_EINTERNAL, "update row missing from the parent front"};
          cmap[ro + T.k[t] + q] = pp;
        }
      else if (T.m[t] != 0)
        throw HzError{HZ_EINTERNAL, "root front with update rows"};
      for (int32_t c : T.children[t]) child_idx.push_back(base[i] + c);
      child_ptr[g + 1] = (int)child_idx.size();
      // lower-triangle entries (in elimination order) of the pivot columns
      for (int cj = 0; cj < T.k[t]; ++cj) {
        const int32_t v = T.perm[T.piv_begin[t] + cj];
        for (int64_t p = A.rowptr[v]; p < A.rowptr[v + 1]; ++p) {
          const int32_t r = A.col[p];
          if (T.pos[r] < T.pos[v]) continue;
          int rp = front_pos(t, r);
          if (rp < 0) throw HzError{HZ_EINTERNAL, "matrix entry outside its front"};
          amap_pos.push_back(rp + cj * f[g]);
          amap_val.push_back(aoff + p);
        }
      }
      amap_ptr[g + 1] = (int64_t)amap_pos.size();
    }
  }
  // per-row front id and local position; extend-add sources of every row
  std::vector<int> row_front(rowoff[nf]), row_local(rowoff[nf]);
  for (int g = 0; g < nf; ++g)
    for (int r = 0; r < f[g]; ++r) {
      row_front[rowoff[g] + r] = g;
      row_local[rowoff[g] + r] = r;
    }
  std::vector<std::pair<int64_t, int64_t>> contrib;  // (parent row, child update row), child-list order
  for (int g = 0; g < nf; ++g)
    for (int q = child_ptr[g]; q < child_ptr[g + 1]; ++q) {
      const int ch = child_idx[q];
      for (int a = 0; a < f[ch] - k[ch]; ++a) {
        const int64_t cr = rowoff[ch] + k[ch] + a;
        contrib.push_back({rowoff[g] + cmap[cr], cr});
      }
    }
  std::stable_sort(contrib.begin(), contrib.end(),
                   [](const std::pair<int64_t, int64_t>& x, const std::pair<int64_t, int64_t>& y) {
                     return x.first < y.first;
                   });
  std::vector<int64_t> cptr(rowoff[nf] + 1, 0);
  std::vector<int> cidx(contrib.size());
  for (size_t q = 0; q < contrib.size(); ++q) {
    cptr[contrib[q].first + 1]++;
    cidx[q] = (int)contrib[q].second;
  }
  for (int64_t r = 0; r < rowoff[nf]; ++r) cptr[r + 1] += cptr[r];
  // sweep tiles: (front, first output row, first reduction index, partial slot)
  // and row blocks (front, first output row, tiles, first slot); slots restart
  // at 0 on every level
  std::vector<int4> ftiles, frb, btiles, brb;
  info.ftile_ptr.assign(1, 0);
  info.btile_ptr.assign(1, 0);
  info.frb_ptr.assign(1, 0);
  info.brb_ptr.assign(1, 0);
  // tensor-core mode: eligible tiles go to the tcgen05 kernel with their factor
  // block packed (TF32 planes, K-major core matrices), the rest to the SIMT kernel
  std::vector<int4> fs, bsl, ftc, btc;
  std::vector<int64_t> ftc_off, btc_off;
  int64_t tc_bytes = 0;
  info.fs_ptr.assign(1, 0);
  info.bs_ptr.assign(1, 0);
  info.ftc_ptr.assign(1, 0);
  info.btc_ptr.assign(1, 0);
  auto classify = [&](bool fwd, const int4& tile) {
    const int g = tile.x, r0 = tile.y, c0 = tile.z;
    const int nout = fwd ? f[g] : k[g];
    const int kend = fwd ? (r0 < k[g] ? std::min(k[g], r0 + MF_TILE_ROWS) : k[g]) : f[g];
    const int kbeg = fwd ? c0 : std::max(c0, r0);
    const int kstop = std::min(kend, c0 + MF_TILE_K);
    const int nr = std::min(MF_TILE_ROWS, nout - r0), nk = kstop - kbeg;
    if (tc && nr >= TC_MIN_ROWS && nk >= TC_MIN_K) {
      (fwd ? ftc : btc).push_back(tile);
      (fwd ? ftc_off : btc_off).push_back(tc_bytes);
      tc_bytes += tc_tile_bytes(nr, nk);
    } else {
      (fwd ? fs : bsl).push_back(tile);
    }
  };
  info.fwd_cmacs.assign(maxh + 1, 0.0);
  info.fhalf.assign(maxh + 1, 1);
  info.bhalf.assign(maxh + 1, 1);
  info.bwd_cmacs.assign(maxh + 1, 0.0);
  int64_t max_slots = 1;
  for (int l = 0; l <= maxh; ++l) {
    int fslot = 0, bslot = 0;
    for (int q = info.level_ptr[l]; q < info.level_ptr[l + 1]; ++q) {
      const int g = level_list[q];
      // a row block covered by a single tile finishes inside the tile (slot
      // -1); the others sum their partial tiles in k_mf_reduce. A front
      // without pivots (k = 0) still passes its children's updates on: its
      // row blocks get one tile with an empty reduction
      for (int r0 = 0; r0 < f[g]; r0 += MF_TILE_ROWS) {
        if (f[g] - r0 > 64) info.fhalf[l] = 0;
        const int kend = r0 < k[g] ? std::min(k[g], r0 + MF_TILE_ROWS) : k[g];
        const int nk = (kend + MF_TILE_K - 1) / MF_TILE_K;
        if (nk <= 1) {
          ftiles.push_back(make_int4(g, r0, 0, -1));
          classify(true, ftiles.back());
          continue;
        }
        frb.push_back(make_int4(g, r0, nk, fslot));
        for (int c0 = 0; c0 < kend; c0 += MF_TILE_K) {
          ftiles.push_back(make_int4(g, r0, c0, fslot++));
          classify(true, ftiles.back());
        }
      }
      for (int j0 = 0; j0 < k[g]; j0 += MF_TILE_ROWS) {
        if (k[g] - j0 > 64) info.bhalf[l] = 0;
        const int nk = (f[g] - j0 + MF_TILE_K - 1) / MF_TILE_K;
        if (nk == 1) {
          btiles.push_back(make_int4(g, j0, j0, -1));
          classify(false, btiles.back());
          continue;
        }
        brb.push_back(make_int4(g, j0, nk, bslot));
        for (int c0 = j0; c0 < f[g]; c0 += MF_TILE_K) {
          btiles.push_back(make_int4(g, j0, c0, bslot++));
          classify(false, btiles.back());
        }
      }
      const double kk = k[g], mm = f[g] - k[g];
      info.fwd_cmacs[l] += kk * (kk + 1) / 2 + kk * mm;
      info.bwd_cmacs[l] += kk * (kk + 1) / 2 + kk * mm;
    }
    max_slots = std::max<int64_t>(max_slots, std::max(fslot, bslot));
    info.ftile_ptr.push_back((int)ftiles.size());
    info.btile_ptr.push_back((int)btiles.size());
    info.frb_ptr.push_back((int)frb.size());
    info.brb_ptr.push_back((int)brb.size());
    info.fs_ptr.push_back((int)fs.size());
    info.bs_ptr.push_back((int)bsl.size());
    info.ftc_ptr.push_back((int)ftc.size());
    info.btc_ptr.push_back((int)btc.size());
  }
  info.level_row.assign(maxh + 2, 0);
  for (int l = 0; l <= maxh; ++l) {
    int64_t e = info.level_row[l];
    for (int q = info.level_ptr[l]; q < info.level_ptr[l + 1]; ++q) e += f[level_list[q]];
    info.level_row[l + 1] = e;
  }
  mf.nfronts = nf;
  mf.nlevels = info.nlevels;
  mf.max_f = info.max_front;
  mf.rows_total = rowoff[nf];
  mf.F_total = Foff[nf];
  mf.amap_total = (int64_t)amap_pos.size();
  mf.level_ptr_h = info.level_ptr.data();
  mf.ftile_ptr_h = info.ftile_ptr.data();
  mf.fhalf_h = info.fhalf.data();
  mf.bhalf_h = info.bhalf.data();
  mf.btile_ptr_h = info.btile_ptr.data();
  mf.frb_ptr_h = info.frb_ptr.data();
  mf.brb_ptr_h = info.brb_ptr.data();
  mf.level_row_h = info.level_row.data();
  mf.max_slots = max_slots;
  if (persistent) {
    // the same tiles renumbered for one launch per sweep: slots unique over all levels, the
    // backward tiles ordered from the roots down
    std::vector<int4> ptf, ptb, prbf, prbb;
    std::vector<int> srf, srb, nrbf(nf, 0), nrbb(nf, 0), nch(nf);
    for (int g = 0; g < nf; ++g) nch[g] = child_ptr[g + 1] - child_ptr[g];
    auto renumber = [&](const std::vector<int4>& tl, const std::vector<int>& tptr, bool fwd, std::vector<int4>& out,
                        std::vector<int4>& rbs, std::vector<int>& slot_rb, std::vector<int>& nrb) {
      for (int li = 0; li <= maxh; ++li) {
        const int l = fwd ? li : maxh - li;
        // within a level, tiles of one row block are adjacent (built that way above)
        for (int q = tptr[l]; q < tptr[l + 1]; ++q) {
          int4 t = tl[q];
          if (t.w < 0) {
            out.push_back(t);
            nrb[t.x]++;
            continue;
          }
          const bool first = out.empty() || out.back().w < 0 || out.back().x != t.x || out.back().y != t.y;
          if (first) {
            rbs.push_back(make_int4(t.x, t.y, 0, (int)slot_rb.size()));
            nrb[t.x]++;
          }
          rbs.back().z++;
          t.w = (int)slot_rb.size();
          slot_rb.push_back((int)rbs.size() - 1);
          out.push_back(t);
        }
      }
    };
    renumber(ftiles, info.ftile_ptr, true, ptf, prbf, srf, nrbf);
    renumber(btiles, info.btile_ptr, false, ptb, prbb, srb, nrbb);
    // forward: a front waits for its children that have rows (a child without rows has no update
    // rows either and contributes nothing); backward: a front waits for its nearest ancestor with
    // pivots, which finishes only after all of its own ancestors
    std::vector<int> bdep(nf, -1);
    for (int g = 0; g < nf; ++g) {
      nch[g] = 0;
      for (int q = child_ptr[g]; q < child_ptr[g + 1]; ++q) nch[g] += nrbf[child_idx[q]] > 0;
      int a = parent[g];
      while (a >= 0 && nrbb[a] == 0) a = parent[a];
      bdep[g] = a;
    }
    mf.persistent = 1;
    mf.pt_nf = (int)ptf.size();
    mf.pt_nb = (int)ptb.size();
    mf.prb_nf = (int)prbf.size();
    mf.prb_nb = (int)prbb.size();
    mf.ptf = pool.upload(ptf, st);
    mf.ptb = pool.upload(ptb, st);
    mf.slot_rb_f = pool.upload(srf, st);
    mf.slot_rb_b = pool.upload(srb, st);
    mf.prb_f = pool.upload(prbf, st);
    mf.prb_b = pool.upload(prbb, st);
    mf.nrb_f = pool.upload(nrbf, st);
    mf.nrb_b = pool.upload(nrbb, st);
    mf.parent = pool.upload(parent, st);
    mf.bdep = pool.upload(bdep, st);
    mf.nchild = pool.upload(nch, st);
    mf.cnt_n = 1 + std::max(mf.prb_nf, mf.prb_nb) + 2 * nf;
    mf.cnt = pool.alloc<int>(mf.cnt_n);
    mf.pslots = std::max<int64_t>(1, std::max(srf.size(), srb.size()));
    mf.sw_err = pool.alloc<int>(1);
    CK(cudaMemsetAsync(mf.sw_err, 0, sizeof(int), st));
  }
  mf.frb = pool.upload(frb, st);
  mf.brb = pool.upload(brb, st);
  mf.row_front = pool.upload(row_front, st);
  mf.row_local = pool.upload(row_local, st);
  mf.cptr = pool.upload(cptr, st);
  mf.cidx = pool.upload(cidx, st);
  mf.cidx_n = (int64_t)cidx.size();
  mf.ftiles_n = (int64_t)ftiles.size();
  mf.btiles_n = (int64_t)btiles.size();
  mf.fp32 = fp32 ? 1 : 0;
  mf.M_total = Moff[nf];
  mf.D_total = Doff[nf];
  mf.ftiles = pool.upload(ftiles, st);
  mf.btiles = pool.upload(btiles, st);
  mf.Moff = pool.upload(Moff, st);
  mf.Doff = pool.upload(Doff, st);
  const size_t esz = fp32 ? sizeof(float2) : sizeof(double2);
  mf.M = pool.alloc<char>(Moff[nf] * esz);
  mf.MT = pool.alloc<char>(Moff[nf] * esz);
  mf.Dinv = pool.alloc<char>(Doff[nf] * esz);
  mf.level_list = pool.upload(level_list, st);
  mf.k = pool.upload(k, st);
  mf.f = pool.upload(f, st);
  mf.Foff = pool.upload(Foff, st);
  mf.rowoff = pool.upload(rowoff, st);
  mf.rows = pool.upload(rows, st);
  mf.cmap = pool.upload(cmap, st);
  mf.child_ptr = pool.upload(child_ptr, st);
  mf.child_idx = pool.upload(child_idx, st);
  mf.amap_ptr = pool.upload(amap_ptr, st);
  mf.amap_pos = pool.upload(amap_pos, st);
  mf.amap_val = pool.upload(amap_val, st);
  mf.Aval = pool.upload(Aval, st);
  mf.aval_n = (int64_t)Aval.size();
  mf.fr32 = fr32 ? 1 : 0;
  mf.F = fr32 ? (void*)pool.alloc<float2>(Foff[nf]) : (void*)pool.alloc<double2>(Foff[nf]);
  {
    // factorisation schedule: small fronts one CTA each; large ones by panels with tiled trailing updates
    std::vector<int> small, big;
    std::vector<int4> ft, fi;
    std::vector<int64_t> pan_off;
    int64_t pan_total = 0;
    info.fa_small_ptr.assign(1, 0);
    info.fa_big_ptr.assign(1, 0);
    info.fa_step_ptr.assign(1, 0);
    info.fa_tile_ptr.assign(1, 0);
    info.fi_tile_ptr.assign(1, 0);
    for (int l = 0; l <= maxh; ++l) {
      int kmax = 0;
      std::vector<int> lbig;
      for (int q = info.level_ptr[l]; q < info.level_ptr[l + 1]; ++q) {
        const int g = level_list[q];
        if (f[g] <= FA_SMALL) {
          small.push_back(g);
        } else {
          lbig.push_back(g);
          kmax = std::max(kmax, k[g]);
        }
      }
      const int bfirst = (int)big.size();
      big.insert(big.end(), lbig.begin(), lbig.end());
      for (int g : lbig) {
        pan_off.push_back(pan_total);
        pan_total += (int64_t)f[g] * FA_NB_H;
      }
      const int nsteps = lbig.empty() ? 0 : (kmax + FA_NB_H - 1) / FA_NB_H;
      for (int p = 0; p < nsteps; ++p) {
        const int p0 = p * FA_NB_H;
        for (size_t bi = 0; bi < lbig.size(); ++bi) {
          const int g = lbig[bi];
          if (p0 >= k[g]) continue;
          const int q0 = p0 + std::min(FA_NB_H, k[g] - p0);
          const int T = (f[g] - q0 + FA_TILE_H - 1) / FA_TILE_H;
          for (int ti = 0; ti < T; ++ti)
            for (int tj = 0; tj <= ti; ++tj) ft.push_back(make_int4(g, ti, tj, 0));
          // inverse: rows below the block x columns [0, q0); w = the front's index in the level's big list
          const int Tc = (q0 + FA_TILE_H - 1) / FA_TILE_H;
          for (int ti = 0; ti < T; ++ti)
            for (int tj = 0; tj < Tc; ++tj) fi.push_back(make_int4(g, ti, tj, (int)bi));
        }
        info.fa_tile_ptr.push_back((int)ft.size());
        info.fi_tile_ptr.push_back((int)fi.size());
      }
      (void)bfirst;
      info.fa_small_ptr.push_back((int)small.size());
      info.fa_big_ptr.push_back((int)big.size());
      info.fa_step_ptr.push_back(info.fa_step_ptr.back() + nsteps);
    }
    mf.fa_small = pool.upload(small, st);
    mf.fa_big = pool.upload(big, st);
    mf.fa_tiles = pool.upload(ft, st);
    mf.fi_tiles = pool.upload(fi, st);
    mf.fa_pan_off = pool.upload(pan_off, st);
    mf.fa_pan = fr32 ? (void*)pool.alloc<float2>(std::max<int64_t>(pan_total, 1))
                     : (void*)pool.alloc<double2>(std::max<int64_t>(pan_total, 1));
    mf.fi_tile_ptr_h = info.fi_tile_ptr.data();
    mf.fa_small_ptr_h = info.fa_small_ptr.data();
    mf.fa_big_ptr_h = info.fa_big_ptr.data();
    mf.fa_step_ptr_h = info.fa_step_ptr.data();
    mf.fa_tile_ptr_h = info.fa_tile_ptr.data();
  }
  mf.perturbed = pool.alloc<int>(1);
  CK(cudaMemsetAsync(mf.perturbed, 0, sizeof(int), st));
  mf.tc = tc ? 1 : 0;
  if (tc) {
    mf.fs_ptr_h = info.fs_ptr.data();
    mf.bs_ptr_h = info.bs_ptr.data();
    mf.ftc_ptr_h = info.ftc_ptr.data();
    mf.btc_ptr_h = info.btc_ptr.data();
    mf.ftiles_s = pool.upload(fs, st);
    mf.btiles_s = pool.upload(bsl, st);
    mf.ftiles_tc = pool.upload(ftc, st);
    mf.btiles_tc = pool.upload(btc, st);
    mf.ftc_off = pool.upload(ftc_off, st);
    mf.btc_off = pool.upload(btc_off, st);
    mf.ftc_n = (int64_t)ftc.size();
    mf.btc_n = (int64_t)btc.size();
    mf.tc_bytes = tc_bytes;
    mf.TC = pool.alloc<unsigned char>((size_t)std::max<int64_t>(tc_bytes, 16));
    mf.tc_err = pool.alloc<int>(1);
    CK(cudaMemsetAsync(mf.tc_err, 0, sizeof(int), st));
    CK(cudaStreamCreateWithFlags(&mf.side, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&mf.ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&mf.ev_join, cudaEventDisableTiming));
  }
}

void destroy_side(DevMF& mf) {
  if (mf.side) {
    cudaStreamSynchronize(mf.side);
    cudaStreamDestroy(mf.side);
  }
  if (mf.ev_fork) cudaEventDestroy(mf.ev_fork);
  if (mf.ev_join) cudaEventDestroy(mf.ev_join);
  mf.side = nullptr;
  mf.ev_fork = mf.ev_join = nullptr;
}

// (hi, lo) pairs of FP32 numbers with hi + lo = v to about 48 bits
static std::vector<float2> df_pairs(const std::vector<double>& v) {
  std::vector<float2> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) {
    const float h = (float)v[i];
    o[i] = make_float2(h, (float)(v[i] - (double)h));
  }
  return o;
}

void upload_split_df(const CsrC& A, DevSplitCsr& D, DevPool& pool, cudaStream_t st) {
  CsrR re, im;
  split_re_im(A, re, im);
  D.val_re_df = pool.upload(df_pairs(re.val), st);
  D.val_im_df = pool.upload(df_pairs(im.val), st);
}

void upload_split(const CsrC& A, DevSplitCsr& D, DevPool& pool, cudaStream_t st, bool with_f32 = false,
                  bool with_df = false) {
  CsrR re, im;
  split_re_im(A, re, im);
  if (with_f32) {
    std::vector<float> rf(re.val.begin(), re.val.end()), imf(im.val.begin(), im.val.end());
    D.val_re_f = pool.upload(rf, st);
    D.val_im_f = pool.upload(imf, st);
  }
  if (with_df) {
    D.val_re_df = pool.upload(df_pairs(re.val), st);
    D.val_im_df = pool.upload(df_pairs(im.val), st);
  }
  D.n = A.nrows;
  D.ncols = A.ncols;
  D.nnz_re = (int64_t)re.col.size();
  D.nnz_im = (int64_t)im.col.size();
  D.rp_re = pool.upload(re.rowptr, st);
  D.col_re = pool.upload(re.col, st);
  D.val_re = pool.upload(re.val, st);
  D.rp_im = pool.upload(im.rowptr, st);
  D.col_im = pool.upload(im.col, st);
  D.val_im = pool.upload(im.val, st);
}

struct DevReal {
  int64_t n = 0, nnz = 0;
  int64_t* rp = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
  float* val_f = nullptr;    // FP32 copy (mixed form)
  float2* val_df = nullptr;  // double-float copy (mixed form, emulate_fp64)
};
void upload_real(const CsrR& A, DevReal& D, DevPool& pool, cudaStream_t st, bool with_f32 = false,
                 bool with_df = false) {
  D.n = A.nrows;
  D.nnz = (int64_t)A.col.size();
  D.rp = pool.upload(A.rowptr, st);
  D.col = pool.upload(A.col, st);
  D.val = pool.upload(A.val, st);
  if (with_f32) {
    std::vector<float> vf(A.val.begin(), A.val.end());
    D.val_f = pool.upload(vf, st);
  }
  if (with_df) D.val_df = pool.upload(df_pairs(A.val), st);
}

struct LevelDev {             // one level of ORAS on the device
  DevMF mf;
  MFHost info;
  int64_t n = 0, sub_rows = 0;
  std::vector<FrontTree> trees;
  double amax = 0.0;
};

void build_level(const Space& sp, const std::vector<Subdomain>& subs, int leaf, bool fp32, bool fr32, bool tc,
                 bool persistent, LevelDev& L, DevPool& pool, cudaStream_t st) {
  const size_t np = subs.size();
  std::vector<int64_t> sub_off(np + 1, 0);
  for (size_t i = 0; i < np; ++i) sub_off[i + 1] = sub_off[i] + (int64_t)subs[i].dofs.size();
  if (sub_off[np] >= (int64_t)1 << 31) throw HzError{HZ_EINVAL, "subdomain rows exceed 2^31"};
  L.n = sp.n;
  L.sub_rows = sub_off[np];
  L.trees.resize(np);
  std::vector<const CsrC*> mats(np);
  std::vector<const FrontTree*> tr(np);
#pragma omp parallel for schedule(dynamic, 1)
  for (long i = 0; i < (long)np; ++i) {
    std::vector<double> X(3 * subs[i].dofs.size());
    for (size_t l = 0; l < subs[i].dofs.size(); ++l)
      for (int d = 0; d < 3; ++d) X[3 * l + d] = sp.coords[3 * subs[i].dofs[l] + d];
    L.trees[i] = nd_symbolic(subs[i].A, X, leaf);
  }
  for (size_t i = 0; i < np; ++i) {
    mats[i] = &subs[i].A;
    tr[i] = &L.trees[i];
    for (const cplx& v : subs[i].A.val) L.amax = std::max(L.amax, std::abs(v));
  }
  build_mf(mats, tr, sub_off, fp32, fr32, tc, persistent, L.mf, L.info, pool, st);
  std::vector<int> gidx(sub_off[np]), own(sp.n, -1);
  for (size_t i = 0; i < np; ++i)
    for (size_t l = 0; l < subs[i].dofs.size(); ++l) {
      gidx[sub_off[i] + l] = (int)subs[i].dofs[l];
      if (subs[i].owned[l]) own[subs[i].dofs[l]] = (int)(sub_off[i] + l);
    }
  for (int64_t g = 0; g < sp.n; ++g)
    if (own[g] < 0) throw HzError{HZ_EINTERNAL, "dof without owning subdomain"};
  L.mf.nsub_rows = sub_off[np];
  L.mf.gidx = pool.upload(gidx, st);
  L.mf.own = pool.upload(own, st);
}

// A single "subdomain" covering the whole matrix: direct factorisation.
void build_direct(const Space& sp, const CsrC& A, int leaf, bool fp32, bool tc, bool persistent, LevelDev& L,
                  DevPool& pool, cudaStream_t st) {  // the coarse factors: factorised in FP64
  std::vector<Subdomain> one(1);
  one[0].dofs.resize(sp.n);
  std::iota(one[0].dofs.begin(), one[0].dofs.end(), 0);
  one[0].owned.assign(sp.n, 1);
  one[0].A = A;
  build_level(sp, one, leaf, fp32, false, tc, persistent, L, pool, st);
}

void mesh_from_abi(const hz_mesh* in, Mesh& m) {
  if (!in || !in->xyz || !in->tets || in->nv <= 0 || in->ne <= 0) throw HzError{HZ_EINVAL, "empty or NULL mesh"};
  if (in->nbf < 0 || (in->nbf > 0 && (!in->bfaces || !in->bface_tag)))
    throw HzError{HZ_EINVAL, "boundary face arrays missing"};
  if (in->nv >= (int64_t)1 << 31) throw HzError{HZ_EINVAL, "too many vertices"};
  m.nv = in->nv;
  m.ne = in->ne;
  m.xyz.assign(in->xyz, in->xyz + 3 * in->nv);
  m.tets.assign(in->tets, in->tets + 4 * in->ne);
  m.bfaces.assign(in->bfaces, in->bfaces + 3 * in->nbf);
  m.btag.assign(in->bface_tag, in->bface_tag + in->nbf);
  for (int32_t v : m.bfaces)
    if (v < 0 || v >= m.nv) throw HzError{HZ_EINVAL, "boundary face vertex out of range"};
}

}  // namespace

enum Phase { PH_SPMM = 0, PH_FRONTS, PH_RESTRICT, PH_COARSE, PH_ARNOLDI, PH_PSPMM, PH_COUNT };
static const char* PHASE_NAMES[PH_COUNT] = {"spmm_A", "fronts", "restrict_prolong", "coarse", "arnoldi",
                                            "precond_spmm"};

// CUDA-event timing of hot-path phases (off unless hz_profile_begin)
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  struct Rec {
    int ph;
    cudaEvent_t a, b;
    double flops, bytes;
  };
  std::vector<Rec> recs;
  cudaEvent_t ev() {
    if (used == pool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) throw HzError{HZ_ECUDA, "cudaEventCreate failed"};
      pool.push_back(e);
    }
    return pool[used++];
  }
  int begin(int ph, cudaStream_t st) {
    if (!on) return -1;
    Rec r{ph, ev(), ev(), 0.0, 0.0};
    CK(cudaEventRecord(r.a, st));
    recs.push_back(r);
    return (int)recs.size() - 1;
  }
  void end(int id, cudaStream_t st, double flops, double bytes) {
    if (id < 0) return;
    CK(cudaEventRecord(recs[id].b, st));
    recs[id].flops = flops;
    recs[id].bytes = bytes;
  }
  void destroy() {
    for (auto e : pool) cudaEventDestroy(e);
    pool.clear();
  }
};

// A captured CUDA graph of a fixed launch sequence, re-captured when the
// block width or the workspace changes.
struct GraphCache {
  int s = -1;
  long long kernels = 0;  // kernel launches recorded in the graph
  cudaGraphExec_t exec = nullptr;
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    s = -1;
  }
};

struct hz_ctx {
  hz_options opt;
  Profiler prof;
  cudaStream_t st = nullptr;       // the library's own stream (graph capture needs a non-default stream)
  cudaStream_t user_st = nullptr;  // the caller's stream: every call first waits for its pending work
  cudaEvent_t ev_join = nullptr;
  GraphCache g_fronts, g_coarse;
  DevPool pool;
  Mesh fine, coarse;
  Space space;
  CsrC A_host;
  DevSplitCsr A;
  LevelDev lf;                // fine ORAS level
  bool has_coarse = false;
  bool coarse32 = false;      // mixed form with coarse_fp32: the whole of M^{-1} on FP32 blocks
  bool df = false;            // mixed form with emulate_fp64: products with A and E in double-float
  float4 *Xdf = nullptr, *XdfH = nullptr;  // double-float copies of the product's input block (fine, coarse)
  Space cspace;
  DevSplitCsr E;
  DevReal Z, ZT;
  LevelDev lc;                // coarse ORAS level (or direct factors of E)
  int perturbed = 0;
  double setup_s = 0, factor_s = 0;
  int device = -1;                 // the device hz_setup ran on
  void* noalloc_scratch = nullptr; // device address of the allocation-free product's scratch
  // per-column results of the last solve call (hz_column_stats)
  std::vector<double> col_res;
  std::vector<int> col_its;
  // workspaces (capacity s_cap columns)
  int s_cap = 0;
  DevPool work;
  double2 *B = nullptr, *X = nullptr, *R = nullptr, *T = nullptr, *Q = nullptr, *Xsub = nullptr, *U = nullptr;
  double2 *rH = nullptr, *yH = nullptr, *XsubH = nullptr;
  float2 *rH32 = nullptr, *yH32 = nullptr;
  float2 *v32 = nullptr, *q32 = nullptr, *t32 = nullptr;  // FP32 preconditioner blocks (mixed form)
  DevKrylov Kout, Kin;
  DevBlockKrylov Bk;          // block FGMRES (option block_arnoldi), on Kout's basis arrays
  // Krylov subspace recycling (option recycle): rk_eff vectors U, C = A U (orthonormal), [n][rk_eff]
  int rk_eff = 0;
  double2 *Ur = nullptr, *Cr = nullptr, *Un = nullptr, *Cn = nullptr, *Rt1 = nullptr, *Rt2 = nullptr;
  double2 *Rsm = nullptr, *Rp = nullptr;   // device k x k factors / coefficients (small)
  double2 *Bc = nullptr, *Yr = nullptr, *Rpart = nullptr;  // per block: [m][rk][s], [rk][s], partial sums
  double* bnorm = nullptr;
  double* rnorm = nullptr;
  double* h_res = nullptr;    // pinned host
  int* h_done = nullptr;
  int* d_srcidx = nullptr;
  double2* d_srcval = nullptr;
  int src_cap = 0;
  // per-element data of the FWI gradient (uploaded by the first hz_fwi_gradient call)
  double omega = 0;
  std::vector<double> mvals;
  bool fwi_ready = false;
  int* d_fwi_l2g = nullptr;        // [ne][20], -1 on Dirichlet dofs
  double* d_fwi_vol = nullptr;     // [ne]
  double* d_fwi_farea = nullptr;   // [ne][4], area of Robin faces, 0 elsewhere
  double* d_fwi_m = nullptr;       // [ne]
};

namespace {

void alloc_krylov(DevKrylov& K, int64_t n, int s, int m, DevPool& p, bool fp32, bool df = false) {
  K.n = n;
  K.s = s;
  K.m = m;
  K.fp32 = fp32 ? 1 : 0;
  K.df = (df && !fp32) ? 1 : 0;
  K.nblk = 304;
  if (K.df) {
    K.Wdf = p.alloc<float4>((size_t)n * s);
    K.hdf = p.alloc<float4>((size_t)(m + 1) * s);
  }
  const size_t es = fp32 ? sizeof(float2) : sizeof(double2);
  K.V = p.alloc<char>((size_t)(m + 1) * n * s * es);
  K.Zk = p.alloc<char>((size_t)m * n * s * es);
  K.W = p.alloc<char>((size_t)n * s * es);
  K.H = p.alloc<double2>((size_t)s * (m + 1) * m);
  K.hpart = p.alloc<double2>((size_t)K.nblk * (m + 1) * s);
  K.h1 = p.alloc<double2>((size_t)(m + 1) * s);
  K.h2 = p.alloc<double2>((size_t)(m + 1) * s);
  K.cs = p.alloc<double>((size_t)s * m);
  K.sn = p.alloc<double2>((size_t)s * m);
  K.g = p.alloc<double2>((size_t)s * (m + 1));
  K.y = p.alloc<double2>((size_t)s * m);
  K.beta = p.alloc<double>(s);
  K.res = p.alloc<double>(s);
  K.tol = p.alloc<double>(s);
  K.kc = p.alloc<int>(s);
  K.done = p.alloc<int>(s);
  K.reorth = p.alloc<int>(s);
}

void ensure_workspace(hz_ctx* c, int s) {
  if (s <= c->s_cap) {
    c->Kout.s = s;
    c->Kin.s = s;
    return;
  }
  CK(cudaStreamSynchronize(c->st));
  c->g_fronts.reset();
  c->g_coarse.reset();
  c->work.release();
  if (c->h_res) cudaFreeHost(c->h_res);
  if (c->h_done) cudaFreeHost(c->h_done);
  c->h_res = nullptr;
  c->h_done = nullptr;
  c->s_cap = 0;
  const int64_t n = c->space.n;
  DevPool& p = c->work;
  c->B = p.alloc<double2>(n * s);
  c->X = p.alloc<double2>(n * s);
  c->R = p.alloc<double2>(n * s);
  c->T = p.alloc<double2>(n * s);
  c->Q = p.alloc<double2>(n * s);
  c->U = p.alloc<double2>(n * s);
  const size_t ef = c->lf.mf.fp32 ? sizeof(float2) : sizeof(double2);
  c->Xsub = (double2*)p.alloc<char>(c->lf.sub_rows * s * ef);
  c->lf.mf.Wout = p.alloc<char>(c->lf.mf.rows_total * s * ef);
  c->lf.mf.P = p.alloc<char>((size_t)std::max(c->lf.mf.max_slots, c->lf.mf.pslots) * MF_TILE_ROWS * s * ef);
  c->lf.mf.s_cap = s;
  // double-float Arnoldi for the outer space unless block FGMRES or recycling (which read W in FP64)
  alloc_krylov(c->Kout, n, s, c->opt.restart, p, false,
               c->df && !c->opt.block_arnoldi && c->opt.recycle == 0);
  if (c->df) {
    c->Xdf = p.alloc<float4>(n * s);
    if (c->has_coarse && !c->coarse32) c->XdfH = p.alloc<float4>(c->cspace.n * s);
  }
  if (c->opt.recycle > 0) {
    const int rk = c->opt.recycle, m = c->opt.restart;
    c->Kout.Hraw = p.alloc<double2>((size_t)s * (m + 1) * m);
    c->Bc = p.alloc<double2>((size_t)m * rk * s);
    c->Yr = p.alloc<double2>((size_t)rk * std::max(s, rk));
    c->Rpart = p.alloc<double2>((size_t)c->Kout.nblk * rk * std::max(s, rk));
  }
  if (c->opt.block_arnoldi) {
    DevBlockKrylov& B = c->Bk;
    const int m = c->opt.restart;
    B.m = m;
    B.s = s;
    B.n = n;
    B.nblk = 304;
    B.V = (double2*)c->Kout.V;
    B.Zk = (double2*)c->Kout.Zk;
    B.W = (double2*)c->Kout.W;
    B.Hd = p.alloc<double2>((size_t)(m + 1) * s * m * s);
    B.Gr = p.alloc<double2>((size_t)(m + 1) * s * s);
    B.rc = p.alloc<double>((size_t)m * s * s);
    B.rsn = p.alloc<double2>((size_t)m * s * s);
    B.part = p.alloc<double2>((size_t)B.nblk * (m + 1) * s * s);
    B.h1 = p.alloc<double2>((size_t)(m + 1) * s * s);
    B.h2 = p.alloc<double2>((size_t)(m + 1) * s * s);
    B.gram = p.alloc<double2>((size_t)s * s);
    B.R = p.alloc<double2>((size_t)s * s);
    B.Racc = p.alloc<double2>((size_t)s * s);
    B.Y = p.alloc<double2>((size_t)s * m * s);
    B.res = c->Kout.res;
    B.tol = c->Kout.tol;
    B.done = c->Kout.done;
    B.kb = p.alloc<int>(1);
    B.deflated = p.alloc<int>(1);
  }
  if (c->has_coarse) {
    const int64_t nh = c->cspace.n;
    c->rH = p.alloc<double2>(nh * s);
    c->yH = p.alloc<double2>(nh * s);
    const size_t ec = c->lc.mf.fp32 ? sizeof(float2) : sizeof(double2);
    c->XsubH = (double2*)p.alloc<char>(c->lc.sub_rows * s * ec);
    c->lc.mf.Wout = p.alloc<char>(c->lc.mf.rows_total * s * ec);
    c->lc.mf.P = p.alloc<char>((size_t)std::max(c->lc.mf.max_slots, c->lc.mf.pslots) * MF_TILE_ROWS * s * ec);
    c->lc.mf.s_cap = s;
    if (c->opt.coarse_mode == HZ_COARSE_GMRES) {
      alloc_krylov(c->Kin, nh, s, std::max(1, c->opt.coarse_inner_its), p, c->coarse32, c->df);
      CK(cudaMemsetAsync(c->Kin.tol, 0, s * sizeof(double), c->st));
    }
    if (c->coarse32) {
      c->rH32 = p.alloc<float2>(nh * s);
      c->yH32 = p.alloc<float2>(nh * s);
      c->v32 = p.alloc<float2>(n * s);
      c->q32 = p.alloc<float2>(n * s);
      c->t32 = p.alloc<float2>(n * s);
    }
  }
  c->bnorm = p.alloc<double>(s);
  c->rnorm = p.alloc<double>(s);
  CK(cudaMallocHost(&c->h_res, 2 * s * sizeof(double)));
  CK(cudaMallocHost(&c->h_done, s * sizeof(int)));
  c->s_cap = s;
}

// Replay `body` (a fixed launch sequence on st) through a captured graph.
template <typename F>
void run_graph(GraphCache* g, int s, cudaStream_t st, F&& body) {
  if (!g) {
    body();
    return;
  }
  if (g->s != s || !g->exec) {
    g->reset();
    cudaGraph_t graph;
    const long long before = g_kernel_launches.load();
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    body();
    CK(cudaStreamEndCapture(st, &graph));
    g->kernels = g_kernel_launches.load() - before;
    count_launch(-g->kernels);  // captured, not executed
    cudaError_t e = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) throw CudaFail{e, "cudaGraphInstantiate"};
    g->s = s;
  }
  CK(cudaGraphLaunch(g->exec, st));
  count_launch(g->kernels);
}

// ORAS on one level: Z = sum_i R_i^T D_i A_i^{-1} R_i V (+ Qadd)
void apply_oras(LevelDev& L, const double2* V, double2* Zout, const double2* Qadd, double2* Xsub, int s,
                cudaStream_t st, Profiler* prof = nullptr, GraphCache* graph = nullptr) {
  const double es = L.mf.fp32 ? 8.0 : 16.0;
  // gather: indices + read V rows + write sub-vector; scatter: owner index + read + (q) + write
  const double rbytes = 4.0 * L.sub_rows + (16.0 + es) * L.sub_rows * s + 4.0 * L.n +
                        (es + 16.0 + (Qadd ? 16.0 : 0.0)) * L.n * s;
  const double fbytes = es * 2.0 * L.info.factor_entries + 2.0 * es * s * L.sub_rows;
  const double fflops = 8.0 * s * 2.0 * L.info.factor_entries;
  int p0 = prof ? prof->begin(PH_RESTRICT, st) : -1;
  if (L.mf.fp32)
    gather_rows_f32(L.mf.gidx, L.sub_rows, V, (float2*)Xsub, s, st);
  else
    gather_rows(L.mf.gidx, L.sub_rows, V, Xsub, s, st);
  if (prof) prof->end(p0, st, 0.0, 0.0);
  int p1 = prof ? prof->begin(PH_FRONTS, st) : -1;
  run_graph(graph, s, st, [&]() { mf_solve(L.mf, Xsub, s, st); });
  if (prof) prof->end(p1, st, fflops, fbytes);
  int p2 = prof ? prof->begin(PH_RESTRICT, st) : -1;
  if (L.mf.fp32)
    scatter_owned_f32(L.mf.own, L.n, (const float2*)Xsub, Qadd, Zout, s, st);
  else
    scatter_owned(L.mf.own, L.n, Xsub, Qadd, Zout, s, st);
  if (prof) prof->end(p2, st, 0.0, rbytes);
}

// y_H ~ E^{-1} r_H: a fixed number of right-preconditioned GMRES steps on E
// with one-level ORAS on the coarse mesh (or the direct factors of E). In the
// mixed form the whole inner iteration runs on FP32 blocks.
void coarse_solve(hz_ctx* c, const double2* rH, double2* yH, int s) {
  cudaStream_t st = c->st;
  const int64_t nh = c->cspace.n;
  LevelDev& L = c->lc;
  if (c->opt.coarse_mode == HZ_COARSE_DIRECT) {
    apply_oras(L, rH, yH, nullptr, c->XsubH, s, st);
    return;
  }
  DevKrylov& K = c->Kin;
  K.s = s;
  const int64_t vs = nh * s;
  if (K.fp32) {
    float2* V = (float2*)K.V;
    float2* Zk = (float2*)K.Zk;
    float2* Xs = (float2*)c->XsubH;
    if (rH) cast_d2f(rH, c->rH32, vs, st);
    CK(cudaMemsetAsync(c->yH32, 0, vs * sizeof(float2), st));
    krylov_start(K, c->rH32, st);
    for (int j = 0; j < K.m; ++j) {
      gather_rows_ff(L.mf.gidx, L.sub_rows, V + j * vs, Xs, s, st);
      mf_solve(L.mf, Xs, s, st);
      scatter_owned_ff(L.mf.own, L.n, Xs, Zk + j * vs, s, st);
      spmm_split_f32(c->E, Zk + j * vs, (float2*)K.W, s, st);
      krylov_arnoldi(K, j, st);
    }
    krylov_update(K, c->yH32, st);
    if (yH) cast_f2d(c->yH32, yH, vs, st);
    return;
  }
  double2* V = (double2*)K.V;
  double2* Zk = (double2*)K.Zk;
  axpy_cols_zero(yH, vs, st);
  krylov_start(K, rH, st);
  for (int j = 0; j < K.m; ++j) {
    apply_oras(L, V + j * vs, Zk + j * vs, nullptr, c->XsubH, s, st);
    if (c->df) {
      to_df(Zk + j * vs, c->XdfH, vs, st);
      spmm_split_df(c->E, c->XdfH, (double2*)K.W, nullptr, s, 0, st, K.df ? K.Wdf : nullptr);
    } else {
      spmm_split(c->E, Zk + j * vs, (double2*)K.W, nullptr, s, 0, st);
    }
    krylov_arnoldi(K, j, st);
  }
  krylov_update(K, yH, st);
}

// algorithmic cost of Y = A X (split real/imaginary CSR, complex block of s)
static void spmm_cost(const DevSplitCsr& A, int s, bool with_b, double& flops, double& bytes) {
  const double nz = (double)(A.nnz_re + A.nnz_im);
  flops = 4.0 * nz * s;
  bytes = 12.0 * nz + 16.0 * (A.n + 1) + 16.0 * A.ncols * s + 16.0 * A.n * s * (with_b ? 2.0 : 1.0);
}

void spmm_A(hz_ctx* c, const double2* X, double2* Y, const double2* B, int s, int mode) {
  double fl, by;
  spmm_cost(c->A, s, mode == 1, fl, by);
  int id = c->prof.begin(PH_SPMM, c->st);
  if (c->df) {
    to_df(X, c->Xdf, c->space.n * s, c->st);
    spmm_split_df(c->A, c->Xdf, Y, B, s, mode, c->st);
  } else {
    spmm_split(c->A, X, Y, B, s, mode, c->st);
  }
  c->prof.end(id, c->st, fl, by);
}

// A X into a double-float block (the Krylov product of the double-float Arnoldi)
void spmm_A_df(hz_ctx* c, const double2* X, float4* Ydf, int s) {
  double fl, by;
  spmm_cost(c->A, s, false, fl, by);
  int id = c->prof.begin(PH_SPMM, c->st);
  to_df(X, c->Xdf, c->space.n * s, c->st);
  spmm_split_df(c->A, c->Xdf, nullptr, nullptr, s, 0, c->st, Ydf);
  c->prof.end(id, c->st, fl, by);
}

// Algorithmic cost of the coarse phase of one application of M^{-1}: r_H =
// Z^T v, the coarse solve (inner GMRES steps on E with coarse ORAS, or the
// direct factors of E) and q = Z y_H. Bytes: the compulsory traffic of each
// step (matrix and factor entries with their indices, the blocks read and
// written); flops: complex multiply-add = 8 (real-by-complex = 4).
void coarse_cost(const hz_ctx* c, int s, bool f32_input, double& flops, double& bytes) {
  const LevelDev& L = c->lc;
  const double ef = L.mf.fp32 ? 8.0 : 16.0;         // factor and sub-vector entry
  const double es = c->coarse32 ? 8.0 : 16.0;       // block entry (Krylov, E and Z products)
  const double vs = c->coarse32 ? 4.0 : 8.0;        // real matrix value
  const double n = (double)c->space.n, nh = (double)c->cspace.n, sub = (double)L.sub_rows;
  const double nz = (double)c->Z.nnz;
  const double lf = (double)L.info.factor_entries;
  // Z^T v and Z y (+ the FP64 -> FP32 cast of v in the FP32 coarse form)
  bytes = 2.0 * (nz * (vs + 4.0) + 8.0 * (n + 1.0)) + 2.0 * es * s * (n + nh);
  flops = 2.0 * 4.0 * nz * s;
  if (f32_input) bytes += 24.0 * n * s;
  // one application of coarse ORAS (gather, front sweeps, owner scatter)
  const double oras_b = 4.0 * sub + (es + ef) * sub * s + ef * 2.0 * lf + 2.0 * ef * sub * s + 4.0 * nh + (ef + es) * nh * s;
  const double oras_f = 8.0 * s * 2.0 * lf;
  if (c->opt.coarse_mode == HZ_COARSE_DIRECT) {
    bytes += oras_b;
    flops += oras_f;
    return;
  }
  const double nzE = (double)(c->E.nnz_re + c->E.nnz_im);
  const int m = std::max(1, c->opt.coarse_inner_its);
  bytes += 3.0 * es * nh * s;  // Krylov start: norm, scale
  for (int j = 0; j < m; ++j) {
    bytes += oras_b + nzE * (vs + 4.0) + 8.0 * (nh + 1.0) + 2.0 * es * nh * s + es * nh * s * (4.0 * (j + 1) + 6.0);
    flops += oras_f + 4.0 * nzE * s + 2.0 * 2.0 * 8.0 * nh * (j + 1) * s;
  }
  bytes += es * nh * s * (m + 2.0);  // X += Zk y
  flops += 8.0 * nh * s * m;
}

// Zout = M^{-1} V (Eq. 2lvl; Eq. oras without a coarse level)
void apply_prec(hz_ctx* c, const double2* V, double2* Zout, int s) {
  cudaStream_t st = c->st;
  GraphCache* gf = c->opt.use_graphs ? &c->g_fronts : nullptr;
  if (!c->has_coarse) {
    apply_oras(c->lf, V, Zout, nullptr, c->Xsub, s, st, &c->prof, gf);
    return;
  }
  if (c->lf.mf.fp32 && c->v32 && c->opt.coarse_mode == HZ_COARSE_GMRES) {
    // mixed form: the whole of M^{-1} on FP32 blocks, z returned in FP64
    const int64_t n = c->space.n;
    int id = c->prof.begin(PH_COARSE, st);
    cast_d2f(V, c->v32, n * s, st);
    spmm_real_f32(c->ZT.n, c->ZT.rp, c->ZT.col, c->ZT.val_f, c->v32, c->rH32, s, st);  // r_H = Z^T v
    run_graph(c->opt.use_graphs ? &c->g_coarse : nullptr, s, st,
              [&]() { coarse_solve(c, nullptr, nullptr, s); });                         // y_H ~ E^{-1} r_H
    spmm_real_f32(c->Z.n, c->Z.rp, c->Z.col, c->Z.val_f, c->yH32, c->q32, s, st);      // q = Z y_H
    if (id >= 0) {
      double cf, cb;
      coarse_cost(c, s, true, cf, cb);
      c->prof.end(id, st, cf, cb);
    }
    int ip = c->prof.begin(PH_PSPMM, st);
    spmm_split_f32(c->A, c->q32, c->t32, s, st, c->v32);                               // t = v - A q
    c->prof.end(ip, st, 4.0 * (c->A.nnz_re + c->A.nnz_im) * s,
                6.0 * (c->A.nnz_re + c->A.nnz_im) + 16.0 * (n + 1) + 24.0 * n * s);
    LevelDev& L = c->lf;
    int p0 = c->prof.begin(PH_RESTRICT, st);
    gather_rows_ff(L.mf.gidx, L.sub_rows, c->t32, (float2*)c->Xsub, s, st);
    c->prof.end(p0, st, 0.0, 0.0);
    int p1 = c->prof.begin(PH_FRONTS, st);
    run_graph(gf, s, st, [&]() { mf_solve(L.mf, c->Xsub, s, st); });
    c->prof.end(p1, st, 8.0 * s * 2.0 * L.info.factor_entries,
                8.0 * 2.0 * L.info.factor_entries + 2.0 * 8.0 * s * L.sub_rows);
    int p2 = c->prof.begin(PH_RESTRICT, st);
    scatter_owned_fq(L.mf.own, L.n, (const float2*)c->Xsub, c->q32, Zout, s, st);     // z = M1^{-1} t + q
    c->prof.end(p2, st, 0.0, 4.0 * L.sub_rows + 16.0 * L.sub_rows * s + 4.0 * L.n + 32.0 * L.n * s);
    return;
  }
  int id = c->prof.begin(PH_COARSE, st);
  if (c->ZT.val_df) {  // double-float restriction and prolongation
    to_df(V, c->Xdf, c->space.n * s, st);
    spmm_real_df(c->ZT.n, c->ZT.rp, c->ZT.col, c->ZT.val_df, c->Xdf, c->rH, s, st);   // r_H = Z^T v
  } else {
    spmm_real(c->ZT.n, c->ZT.rp, c->ZT.col, c->ZT.val, V, c->rH, s, st);
  }
  run_graph(c->opt.use_graphs ? &c->g_coarse : nullptr, s, st,
            [&]() { coarse_solve(c, c->rH, c->yH, s); });                 // y_H ~ E^{-1} r_H
  if (c->Z.val_df) {
    to_df(c->yH, c->XdfH, c->cspace.n * s, st);
    spmm_real_df(c->Z.n, c->Z.rp, c->Z.col, c->Z.val_df, c->XdfH, c->Q, s, st);       // q = Z y_H
  } else {
    spmm_real(c->Z.n, c->Z.rp, c->Z.col, c->Z.val, c->yH, c->Q, s, st);
  }
  if (id >= 0) {
    double cf, cb;
    coarse_cost(c, s, false, cf, cb);
    c->prof.end(id, st, cf, cb);
  }
  spmm_A(c, c->Q, c->T, V, s, 1);                                         // t = v - A q
  apply_oras(c->lf, c->T, Zout, c->Q, c->Xsub, s, st, &c->prof, gf);      // z = M1^{-1} t + q
}

// One restart cycle of flexible GMRES on the block: Krylov space from the
// current residual c->R, at most max_its iterations (fewer when every column
// has converged or broken down), then X += Zk y. K.tol must hold the
// per-column absolute tolerances. Returns the iterations done.
void check_launch();

int fgmres_cycle(hz_ctx* c, int s, int max_its, bool recyc = false) {
  cudaStream_t st = c->st;
  const int64_t n = c->space.n;
  DevKrylov& K = c->Kout;
  K.s = s;
  const int m = std::min(c->opt.restart, max_its);
  const int64_t vs = n * s;
  const int rk = recyc ? c->rk_eff : 0;  // recycled directions projected out of every A z
  krylov_start(K, c->R, st);
  int its = 0;
  for (int j = 0; j < m; ++j) {
    apply_prec(c, (double2*)K.V + j * vs, (double2*)K.Zk + j * vs, s);
    if (K.df)
      spmm_A_df(c, (double2*)K.Zk + j * vs, K.Wdf, s);
    else
      spmm_A(c, (double2*)K.Zk + j * vs, (double2*)K.W, nullptr, s, 0);
    int id = c->prof.begin(PH_ARNOLDI, st);
    if (rk > 0) {  // B_j = C^H w, w -= C B_j
      double2* Bj = c->Bc + (size_t)j * rk * s;
      recycle_dot(c->Cr, rk, (double2*)K.W, s, n, c->Rpart, K.nblk, Bj, st);
      recycle_axpy(c->Cr, rk, Bj, (double2*)K.W, s, n, -1.0, st);
    }
    krylov_arnoldi(K, j, st);
    // two CGS passes (dots + update) over V_0..j and W, a norm and a scale
    c->prof.end(id, st, 2.0 * 2.0 * 8.0 * n * (j + 1) * s, 16.0 * n * s * (4.0 * (j + 1) + 6.0));
    ++its;
    CK(cudaMemcpyAsync(c->h_done, K.done, s * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    bool alldone = true;
    for (int q = 0; q < s; ++q) alldone &= c->h_done[q] != 0;
    if (alldone) break;
  }
  krylov_update(K, c->X, st);
  if (rk > 0) {  // x -= U sum_j B_j y_j
    recycle_corr(c->Bc, K.y, K.kc, rk, s, K.m, c->Yr, st);
    recycle_axpy(c->Ur, rk, c->Yr, c->X, s, n, -1.0, st);
  }
  return its;
}

// Recycling, start of a cycle: x += U C^H r, r -= C C^H r for every column.
void recycle_project(hz_ctx* c, int s) {
  const int rk = c->rk_eff;
  if (rk == 0) return;
  const int64_t n = c->space.n;
  recycle_dot(c->Cr, rk, c->R, s, n, c->Rpart, c->Kout.nblk, c->Yr, c->st);
  recycle_axpy(c->Ur, rk, c->Yr, c->X, s, n, 1.0, c->st);
  recycle_axpy(c->Cr, rk, c->Yr, c->R, s, n, -1.0, c->st);
}

// Cholesky R^H R = G of a small Hermitian matrix (row-major, k x k); false if
// a pivot is not clearly positive
static bool small_cholesky(const std::vector<double2>& G, int k, std::vector<double2>& R) {
  R.assign((size_t)k * k, make_double2(0.0, 0.0));
  double gmax = 0.0;
  for (int j = 0; j < k; ++j) gmax = std::max(gmax, G[j * k + j].x);
  for (int j = 0; j < k; ++j) {
    double d = G[j * k + j].x;
    for (int q = 0; q < j; ++q) d -= R[q * k + j].x * R[q * k + j].x + R[q * k + j].y * R[q * k + j].y;
    if (!(d > 1e-12 * gmax)) return false;
    const double rjj = std::sqrt(d);
    R[j * k + j] = make_double2(rjj, 0.0);
    for (int l = j + 1; l < k; ++l) {
      cplx v(G[j * k + l].x, G[j * k + l].y);
      for (int q = 0; q < j; ++q) v -= std::conj(cplx(R[q * k + j].x, R[q * k + j].y)) * cplx(R[q * k + l].x, R[q * k + l].y);
      R[j * k + l] = make_double2(v.real() / rjj, v.imag() / rjj);
    }
  }
  return true;
}

// Recycling, end of a cycle: harmonic Ritz vectors of the slowest column's
// cycle give knew new directions U_new = Z P; they join the kept ones (the
// oldest beyond the option's k are dropped) and C = A U is orthonormalised
// by two Cholesky QR passes, U transformed alike. A failed step keeps the
// previous space.
void recycle_update(hz_ctx* c, int s, const std::vector<int>& kc) {
  const int RK = c->opt.recycle, m = c->opt.restart;
  const int64_t n = c->space.n;
  cudaStream_t st = c->st;
  int col = 0;
  for (int q = 1; q < s; ++q)
    if (kc[q] > kc[col]) col = q;
  const int me = kc[col];
  const int knew = std::min(std::max(1, RK / 2), me - 1);
  if (knew < 1) return;
  std::vector<double2> hraw((size_t)(m + 1) * m);
  CK(cudaMemcpyAsync(hraw.data(), c->Kout.Hraw + (size_t)col * (m + 1) * m, hraw.size() * sizeof(double2),
                     cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  std::vector<cplx> Hb((size_t)(me + 1) * me, cplx(0, 0)), P, theta;
  for (int j = 0; j < me; ++j)
    for (int i = 0; i <= std::min(j + 1, me); ++i)
      Hb[i + (size_t)j * (me + 1)] = cplx(hraw[i + (size_t)j * (m + 1)].x, hraw[i + (size_t)j * (m + 1)].y);
  if (!harmonic_ritz(Hb, me, knew, P, theta)) return;
  std::vector<double2> Pd(P.size());
  for (size_t i = 0; i < P.size(); ++i) Pd[i] = make_double2(P[i].real(), P[i].imag());
  CK(cudaMemcpyAsync(c->Rp, Pd.data(), Pd.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
  const int total = std::min(RK, c->rk_eff + knew), kold = total - knew;
  // new directions and their images: Rt1 = Z P, Rt2 = A Rt1 ([n][knew])
  recycle_build((const double2*)c->Kout.Zk, n * s, s, col, c->Rp, me, knew, c->Rt1, knew, 0, n, st);
  spmm_split(c->A, c->Rt1, c->Rt2, nullptr, knew, 0, st);
  recycle_copy(c->Rt1, knew, 0, c->Un, total, 0, knew, n, st);
  recycle_copy(c->Rt2, knew, 0, c->Cn, total, 0, knew, n, st);
  if (kold > 0) {
    recycle_copy(c->Ur, c->rk_eff, 0, c->Un, total, knew, kold, n, st);
    recycle_copy(c->Cr, c->rk_eff, 0, c->Cn, total, knew, kold, n, st);
  }
  for (int pass = 0; pass < 2; ++pass) {
    recycle_dot(c->Cn, total, c->Cn, total, n, c->Rpart, c->Kout.nblk, c->Rsm, st);
    std::vector<double2> G((size_t)total * total), R;
    CK(cudaMemcpyAsync(G.data(), c->Rsm, G.size() * sizeof(double2), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (!small_cholesky(G, total, R)) return;  // keep the previous space
    CK(cudaMemcpyAsync(c->Rsm, R.data(), R.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
    recycle_trsm(c->Cn, n, total, c->Rsm, st);
    recycle_trsm(c->Un, n, total, c->Rsm, st);
  }
  check_launch();
  std::swap(c->Ur, c->Un);
  std::swap(c->Cr, c->Cn);
  c->rk_eff = total;
}

// One restart cycle of block FGMRES (option block_arnoldi): one Krylov space
// for the whole block from the current residual c->R (which it overwrites),
// at most max_its block steps, then X += Z Y. Every column stops together.
int fgmres_cycle_block(hz_ctx* c, int s, int max_its) {
  cudaStream_t st = c->st;
  const int64_t n = c->space.n;
  DevBlockKrylov& B = c->Bk;
  B.s = s;
  const int m = std::min(c->opt.restart, max_its);
  const int64_t vs = n * s;
  int id0 = c->prof.begin(PH_ARNOLDI, st);
  block_krylov_start(B, c->R, st);
  c->prof.end(id0, st, 2.0 * 12.0 * n * s * s, 2.0 * 16.0 * n * s * 4.0);
  int its = 0;
  for (int j = 0; j < m; ++j) {
    apply_prec(c, B.V + j * vs, B.Zk + j * vs, s);
    spmm_A(c, B.Zk + j * vs, B.W, nullptr, s, 0);
    int id = c->prof.begin(PH_ARNOLDI, st);
    block_krylov_arnoldi(B, j, st);
    // two CGS passes (Gram blocks + update) over V_0..j, then CholQR2 (two Gram + triangular solves)
    c->prof.end(id, st, 32.0 * n * s * s * (j + 1) + 24.0 * n * s * s, 16.0 * n * s * (4.0 * (j + 1) + 14.0));
    ++its;
    CK(cudaMemcpyAsync(c->h_done, B.done, s * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    bool alldone = true;
    for (int q = 0; q < s; ++q) alldone &= c->h_done[q] != 0;
    if (alldone) break;
  }
  block_krylov_update(B, c->X, st);
  return its;
}

// True residual R = B - A X and its column norms (host, into c->h_res).
void true_residual(hz_ctx* c, int s) {
  cudaStream_t st = c->st;
  const int64_t n = c->space.n;
  spmm_A(c, c->X, c->R, c->B, s, 1);
  column_norms(c->R, n, s, c->rnorm, c->Kout, st);
  CK(cudaMemcpyAsync(c->h_res, c->rnorm, s * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
}

// Flexible GMRES on the block c->B (n x s, row-major); solution in c->X.
int fgmres(hz_ctx* c, int s, hz_stats* stats) {
  cudaStream_t st = c->st;
  const int64_t n = c->space.n;
  DevKrylov& K = c->Kout;
  K.s = s;
  const int64_t vs = n * s;
  axpy_cols_zero(c->X, vs, st);
  column_norms(c->B, n, s, c->bnorm, K, st);
  std::vector<double> bn(s), tol(s);
  CK(cudaMemcpyAsync(c->h_res, c->bnorm, s * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int q = 0; q < s; ++q) {
    bn[q] = c->h_res[q];
    tol[q] = c->opt.rtol * bn[q];
  }
  CK(cudaMemcpyAsync(K.tol, tol.data(), s * sizeof(double), cudaMemcpyHostToDevice, st));
  cast_copy(c->B, c->R, vs, st);
  int its = 0, restarts = 0;
  bool all_conv = false;
  double maxrel = 0.0;
  std::vector<int> col_its(s, 0), kc(s);
  const bool block = c->opt.block_arnoldi != 0;
  const bool recyc = !block && c->opt.recycle > 0;
  while (true) {
    if (recyc) recycle_project(c, s);
    const int done_its =
        block ? fgmres_cycle_block(c, s, c->opt.maxit - its) : fgmres_cycle(c, s, c->opt.maxit - its, recyc);
    its += done_its;
    if (!block) CK(cudaMemcpyAsync(kc.data(), K.kc, s * sizeof(int), cudaMemcpyDeviceToHost, st));
    true_residual(c, s);  // synchronises the stream
    for (int q = 0; q < s; ++q) col_its[q] += block ? done_its : kc[q];
    if (recyc) recycle_update(c, s, kc);
    all_conv = true;
    maxrel = 0.0;
    for (int q = 0; q < s; ++q) {
      double rel = bn[q] > 0 ? c->h_res[q] / bn[q] : 0.0;
      maxrel = std::max(maxrel, rel);
      all_conv &= rel <= c->opt.rtol;
    }
    if (c->opt.verbose)
      fprintf(stderr, "[hz] fgmres cycle %d its %d max rel residual %.3e\n", restarts, its, maxrel);
    if (all_conv || its >= c->opt.maxit) break;
    ++restarts;
  }
  for (int q = 0; q < s; ++q) {
    c->col_res.push_back(bn[q] > 0 ? c->h_res[q] / bn[q] : 0.0);
    c->col_its.push_back(col_its[q]);
  }
  if (stats) {
    stats->iterations = its;
    stats->restarts = restarts;
    stats->converged = all_conv ? 1 : 0;
    stats->ncols = s;
    stats->max_rel_residual = maxrel;
  }
  return all_conv ? HZ_OK : HZ_ENOTCONV;
}

// Read and clear the device flags that the tensor-core sweep tiles set when
// they give up waiting on one of their barriers; called after every entry
// point that ran the sweeps, so that a timeout is reported by the call in
// which it happened and does not fail later calls.
void check_sweep_flags(hz_ctx* c) {
  for (DevMF* mf : {&c->lf.mf, &c->lc.mf})
    for (int* flag : {mf->tc_err, mf->sw_err})
      if (flag) {
        int e = 0;
        CK(cudaMemcpyAsync(&e, flag, sizeof(int), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        if (e) {
          CK(cudaMemsetAsync(flag, 0, sizeof(int), c->st));
          CK(cudaStreamSynchronize(c->st));
          throw HzError{HZ_EINTERNAL, flag == mf->tc_err ? "tensor-core sweep tile timed out on a barrier"
                                                         : "persistent front sweep timed out on a dependency"};
        }
      }
}

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

template <typename F>
int guarded(F&& f) {
  try {
    return f();
  } catch (const HzError& e) {
    return fail(e.code, e.msg);
  } catch (const CudaFail& e) {
    return fail(HZ_ECUDA, std::string(e.what) + ": " + cudaGetErrorString(e.e));
  } catch (const std::bad_alloc&) {
    return fail(HZ_ENOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(HZ_EINTERNAL, e.what());
  }
}

void check_launch() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw CudaFail{e, "kernel launch"};
}

// debug_bounds: one device pass over the index maps of the hot path
void check_bounds(hz_ctx* c) {
  cudaStream_t st = c->st;
  int* d_err = c->pool.alloc<int>(1);
  const int big = 0x7fffffff;
  CK(cudaMemcpyAsync(d_err, &big, sizeof(int), cudaMemcpyHostToDevice, st));
  std::vector<std::string> names;
  auto chk = [&](const char* nm, const void* a, int64_t count, int stride, int64_t lo, int64_t hi) {
    check_index_range((const int*)a, count, stride, lo, hi, d_err, (int)names.size(), st);
    names.push_back(nm);
  };
  auto chk_csr = [&](const char* nm, const int32_t* col, int64_t nnz, int64_t ncols) { chk(nm, col, nnz, 1, 0, ncols); };
  chk_csr("A columns (real part)", c->A.col_re, c->A.nnz_re, c->A.ncols);
  chk_csr("A columns (imaginary part)", c->A.col_im, c->A.nnz_im, c->A.ncols);
  for (int lev = 0; lev < (c->has_coarse ? 2 : 1); ++lev) {
    LevelDev& L = lev ? c->lc : c->lf;
    const DevMF& mf = L.mf;
    chk(lev ? "coarse R_i map" : "fine R_i map", mf.gidx, mf.nsub_rows, 1, 0, L.n);
    chk(lev ? "coarse owner map" : "fine owner map", mf.own, L.n, 1, 0, mf.nsub_rows);
    chk(lev ? "coarse front rows" : "fine front rows", mf.rows, mf.rows_total, 1, 0, mf.nsub_rows);
    chk(lev ? "coarse extend-add sources" : "fine extend-add sources", mf.cidx, mf.cidx_n, 1, 0, mf.rows_total);
    chk(lev ? "coarse level list" : "fine level list", mf.level_list, mf.nfronts, 1, 0, mf.nfronts);
    chk(lev ? "coarse forward tiles" : "fine forward tiles", mf.ftiles, mf.ftiles_n, 4, 0, mf.nfronts);
    chk(lev ? "coarse backward tiles" : "fine backward tiles", mf.btiles, mf.btiles_n, 4, 0, mf.nfronts);
  }
  if (c->has_coarse) {
    chk_csr("E columns", c->E.col_re, c->E.nnz_re, c->E.ncols);
    chk_csr("Z columns", c->Z.col, c->Z.nnz, c->cspace.n);
    chk_csr("Z^T columns", c->ZT.col, c->ZT.nnz, c->space.n);
  }
  check_launch();
  int h = big;
  CK(cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h != big) throw HzError{HZ_EINTERNAL, "debug_bounds: index out of range in " + names[h]};
}

// order the library stream after the work already queued on the caller's stream
void join_user(hz_ctx* c) {
  CK(cudaEventRecord(c->ev_join, c->user_st));
  CK(cudaStreamWaitEvent(c->st, c->ev_join, 0));
}

}  // namespace

namespace hz {
// accessors for the allocation-free entry point (noalloc.cu)
const DevSplitCsr* ctx_matrix(const hz_ctx* c, int64_t* n) {
  *n = c->space.n;
  return &c->A;
}
void set_last_error(const char* msg) { g_last_error = msg; }
void ctx_noalloc(const hz_ctx* c, int* device, void** scratch) {
  *device = c->device;
  *scratch = c->noalloc_scratch;
}
cudaError_t noalloc_scratch_address(void** out);  // noalloc.cu
}  // namespace hz

extern "C" {

int hz_default_options(hz_options* o) {
  if (!o) return fail(HZ_EINVAL, "NULL options");
  o->precision = HZ_PREC_FP64;
  o->rtol = 1e-6;
  o->maxit = 500;
  o->restart = 30;
  o->max_block = 64;
  o->coarse_mode = HZ_COARSE_GMRES;
  o->coarse_inner_its = 10;
  o->leaf_size = 64;
  o->pivot_tau = 1e-12;
  o->verbose = 0;
  o->use_graphs = 1;
  o->tensor_cores = 0;
  o->overlap = 1;
  o->coarse_fp32 = 0;
  o->debug_bounds = 0;
  o->block_arnoldi = 0;
  o->persistent_sweeps = 0;
  o->factor_fp32 = 1;
  o->recycle = 0;
  o->emulate_fp64 = 1;
  o->coarse_leaf_size = 0;
  return HZ_OK;
}

int hz_setup(const hz_mesh* fine, const double* velocity, double freq_hz, const int32_t* elem_part, int32_t nparts,
             const hz_mesh* coarse, const hz_options* opt, void* stream, hz_ctx** out) {
  if (!out) return fail(HZ_EINVAL, "NULL output pointer");
  *out = nullptr;
  std::unique_ptr<hz_ctx> c(new hz_ctx());
  int rc = guarded([&]() -> int {
    const double t0 = now_s();
    if (opt)
      c->opt = *opt;
    else
      hz_default_options(&c->opt);
    const hz_options& o = c->opt;
    if (!(freq_hz > 0)) throw HzError{HZ_EINVAL, "frequency must be positive"};
    if (!velocity || !elem_part || nparts <= 0) throw HzError{HZ_EINVAL, "velocity / partition missing"};
    if (o.precision != HZ_PREC_FP64 && o.precision != HZ_PREC_MIXED) throw HzError{HZ_EINVAL, "bad precision"};
    if (o.restart < 1 || o.maxit < 1 || o.max_block < 1 || o.max_block > 64 || !(o.rtol > 0) || o.leaf_size < 1)
      throw HzError{HZ_EINVAL, "bad Krylov options"};
    if (o.coarse_mode < 0 || o.coarse_mode > 2) throw HzError{HZ_EINVAL, "bad coarse_mode"};
    if (o.coarse_mode != HZ_COARSE_NONE && !coarse) throw HzError{HZ_EINVAL, "coarse mesh required"};
    if (o.coarse_mode == HZ_COARSE_GMRES && o.coarse_inner_its < 1) throw HzError{HZ_EINVAL, "coarse_inner_its < 1"};
    if (o.overlap < 1 || o.overlap > 16) throw HzError{HZ_EINVAL, "overlap must be in [1, 16]"};
    if (o.block_arnoldi != 0 && (o.block_arnoldi != 1 || o.max_block > 32))
      throw HzError{HZ_EINVAL, "block_arnoldi needs max_block <= 32"};
    if (o.coarse_leaf_size < 0) throw HzError{HZ_EINVAL, "coarse_leaf_size < 0"};
    if (o.recycle < 0 || o.recycle > 16 || (o.recycle > 0 && (o.block_arnoldi || o.restart < 2)))
      throw HzError{HZ_EINVAL, "recycle must be in [0, 16], with per-column FGMRES and restart >= 2"};
    mesh_from_abi(fine, c->fine);
    mesh_build_adjacency(c->fine);
    const int64_t ne = c->fine.ne;
    std::vector<double> mvals(ne);
    for (int64_t e = 0; e < ne; ++e) {
      if (!(velocity[e] > 0) || !std::isfinite(velocity[e])) throw HzError{HZ_EINVAL, "velocity must be > 0"};
      mvals[e] = 1.0 / (velocity[e] * velocity[e]);
    }
    std::vector<int32_t> part(elem_part, elem_part + ne);
    std::vector<int64_t> pc(nparts, 0);
    for (int32_t p : part) {
      if (p < 0 || p >= nparts) throw HzError{HZ_EINVAL, "element partition out of range"};
      pc[p]++;
    }
    for (int64_t v : pc)
      if (v == 0) throw HzError{HZ_EINVAL, "empty subdomain in the partition"};
    const double omega = 2.0 * M_PI * freq_hz;
    c->omega = omega;
    c->mvals = mvals;
    c->user_st = (cudaStream_t)stream;
    CK(cudaGetDevice(&c->device));
    CK(cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking));
    if (o.block_arnoldi) block_krylov_attrs();
    CK(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    join_user(c.get());
    c->space = p3_space(c->fine);
    if (c->space.n >= (int64_t)1 << 31) throw HzError{HZ_EINVAL, "more than 2^31 dofs"};
    c->A_host = assemble_global(c->fine, c->space, mvals, omega);
    const bool mixed = o.precision == HZ_PREC_MIXED;
    c->df = mixed && o.emulate_fp64 != 0;
    upload_split(c->A_host, c->A, c->pool, c->st, mixed);
    std::vector<Subdomain> subs = build_subdomains(c->fine, c->space, part, nparts, mvals, omega, o.overlap);
    const bool tc = mixed && o.tensor_cores != 0;
    const bool pers = o.persistent_sweeps != 0;
    build_level(c->space, subs, o.leaf_size, mixed, mixed && o.factor_fp32 != 0, tc, pers, c->lf, c->pool, c->st);
    subs.clear();
    if (o.coarse_mode != HZ_COARSE_NONE) {
      c->has_coarse = true;
      mesh_from_abi(coarse, c->coarse);
      CoarseSpace C = build_coarse(c->fine, c->space, mvals, part, omega, c->coarse);
      c->cspace = C.space;
      // coarse level in FP64 unless the mixed form asks for an FP32 coarse level
      // the coarse fronts are factorised in FP64 and, in the mixed form, applied in complex FP32 like
      // the fine ones; E, Z and the inner coarse GMRES stay FP64 unless coarse_fp32 asks for FP32
      const bool cf32 = mixed && o.coarse_fp32 != 0;
      c->coarse32 = cf32;
      upload_split(C.E, c->E, c->pool, c->st, cf32 && o.coarse_mode == HZ_COARSE_GMRES,
                   c->df && !cf32 && o.coarse_mode == HZ_COARSE_GMRES);
      upload_real(C.Z, c->Z, c->pool, c->st, cf32, c->df && !cf32);
      upload_real(C.ZT, c->ZT, c->pool, c->st, cf32, c->df && !cf32);
      if (o.coarse_mode == HZ_COARSE_GMRES) {
        std::vector<Subdomain> csubs =
            build_subdomains(c->coarse, c->cspace, C.part, nparts, C.mvals, omega, o.overlap);
        build_level(c->cspace, csubs, o.coarse_leaf_size > 0 ? o.coarse_leaf_size : o.leaf_size, mixed, false, tc,
                    pers, c->lc, c->pool, c->st);
      } else {
        build_direct(c->cspace, C.E, o.coarse_leaf_size > 0 ? o.coarse_leaf_size : o.leaf_size, mixed, tc, pers,
                     c->lc, c->pool, c->st);
      }
    }
    CK(cudaStreamSynchronize(c->st));
    const double t1 = now_s();
    // an FP32 factorisation perturbs pivots below 1e-6 of max|A_i| (FP32 round-off scale), FP64 below pivot_tau
    const double tau_f = (c->lf.mf.fr32 && o.pivot_tau > 0.0) ? std::max(o.pivot_tau, 1e-6) : o.pivot_tau;
    mf_factor(c->lf.mf, tau_f * c->lf.amax, c->st);
    check_launch();
    if (c->has_coarse) {
      mf_factor(c->lc.mf, o.pivot_tau * c->lc.amax, c->st);
      check_launch();
    }
    int pf = 0, pcnt = 0;
    CK(cudaMemcpyAsync(&pf, c->lf.mf.perturbed, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    if (c->has_coarse) CK(cudaMemcpyAsync(&pcnt, c->lc.mf.perturbed, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    c->factor_s = now_s() - t1;
    // the f x f workspaces are only needed by the factorisation
    c->pool.free_one(c->lf.mf.F, c->lf.mf.F_total * (c->lf.mf.fr32 ? sizeof(float2) : sizeof(double2)));
    c->lf.mf.F = nullptr;
    if (c->has_coarse) {
      c->pool.free_one(c->lc.mf.F, c->lc.mf.F_total * (c->lc.mf.fr32 ? sizeof(float2) : sizeof(double2)));
      c->lc.mf.F = nullptr;
    }
    // the assembly maps and local matrix values are only read by the factorisation
    for (DevMF* mf : {&c->lf.mf, &c->lc.mf}) {
      if (!mf->amap_ptr) continue;
      c->pool.free_one(mf->amap_ptr, (mf->nfronts + 1) * sizeof(int64_t));
      c->pool.free_one(mf->amap_pos, std::max<int64_t>(1, mf->amap_total) * sizeof(int));
      c->pool.free_one(mf->amap_val, std::max<int64_t>(1, mf->amap_total) * sizeof(int64_t));
      c->pool.free_one(mf->Aval, std::max<int64_t>(1, mf->aval_n) * sizeof(double2));
      mf->amap_ptr = nullptr;
      mf->amap_pos = nullptr;
      mf->amap_val = nullptr;
      mf->Aval = nullptr;
    }
    // double-float values of A (mixed form, emulate_fp64), once the factorisation workspaces are gone
    if (c->df) upload_split_df(c->A_host, c->A, c->pool, c->st);
    c->perturbed = pf + pcnt;
    if (o.pivot_tau == 0.0 && c->perturbed) throw HzError{HZ_ESINGULAR, "zero pivot in a local factorisation"};
    if (o.debug_bounds) {
      check_bounds(c.get());
    }
    if (o.recycle > 0) {  // recycled space: lives as long as the context (valid for its A)
      const int64_t n = c->space.n, rk = o.recycle;
      c->Ur = c->pool.alloc<double2>(n * rk);
      c->Cr = c->pool.alloc<double2>(n * rk);
      c->Un = c->pool.alloc<double2>(n * rk);
      c->Cn = c->pool.alloc<double2>(n * rk);
      c->Rt1 = c->pool.alloc<double2>(n * rk);
      c->Rt2 = c->pool.alloc<double2>(n * rk);
      c->Rsm = c->pool.alloc<double2>(rk * rk);
      c->Rp = c->pool.alloc<double2>((int64_t)o.restart * rk);
    }
    // address of the allocation-free product's scratch on this device (loads it here)
    hz::noalloc_scratch_address(&c->noalloc_scratch);
    c->setup_s = now_s() - t0;
    if (o.verbose)
      fprintf(stderr, "[hz] setup n=%lld nnz=%lld fronts=%d levels=%d max_front=%d factor %.3fs total %.3fs\n",
              (long long)c->space.n, (long long)c->A_host.col.size(), c->lf.info.nfronts, c->lf.info.nlevels,
              c->lf.info.max_front, c->factor_s, c->setup_s);
    return HZ_OK;
  });
  if (rc != HZ_OK) {
    if (c) {
      if (c->st) cudaStreamSynchronize(c->st);
      for (DevMF* mf : {&c->lf.mf, &c->lc.mf}) destroy_side(*mf);
      c->pool.release();
      if (c->st) cudaStreamDestroy(c->st);
      if (c->ev_join) cudaEventDestroy(c->ev_join);
    }
    return rc;
  }
  *out = c.release();
  return HZ_OK;
}

int hz_ndof(const hz_ctx* c, int64_t* n) {
  if (!c || !n) return fail(HZ_EINVAL, "NULL argument");
  *n = c->space.n;
  return HZ_OK;
}

int hz_dof_coords(const hz_ctx* c, double* xyz) {
  if (!c || !xyz) return fail(HZ_EINVAL, "NULL argument");
  std::memcpy(xyz, c->space.coords.data(), c->space.coords.size() * sizeof(double));
  return HZ_OK;
}

int hz_get_info(const hz_ctx* c, hz_info* info) {
  if (!c || !info) return fail(HZ_EINVAL, "NULL argument");
  std::memset(info, 0, sizeof(*info));
  info->n = c->space.n;
  info->nnz = (int64_t)c->A_host.col.size();
  info->nnz_imag = c->A.nnz_im;
  info->nparts = (int32_t)c->lf.trees.size();
  info->sub_rows = c->lf.sub_rows;
  info->n_coarse = c->has_coarse ? c->cspace.n : 0;
  info->nnz_coarse = c->has_coarse ? c->E.nnz_re : 0;
  info->factor_entries = c->lf.info.factor_entries;
  info->coarse_factor_entries = c->has_coarse ? c->lc.info.factor_entries : 0;
  info->front_entries = c->lf.info.front_entries;
  info->max_front = c->lf.info.max_front;
  info->nfronts = c->lf.info.nfronts;
  info->nlevels = c->lf.info.nlevels;
  info->perturbed_pivots = c->perturbed;
  info->device_bytes = c->pool.bytes + c->work.bytes;
  info->kernel_launches = g_kernel_launches.load();
  info->factor_ldlt_seconds = 1e-3 * (c->lf.mf.factor_ms + c->lc.mf.factor_ms);
  info->factor_inverse_seconds = 1e-3 * (c->lf.mf.inverse_ms + c->lc.mf.inverse_ms);
  return HZ_OK;
}

int hz_column_stats(const hz_ctx* c, double* rel_residual, int32_t* iterations, int32_t cap, int32_t* ncols) {
  if (!c || !ncols || cap < 0) return fail(HZ_EINVAL, "bad argument");
  const int nc = (int)c->col_res.size();
  *ncols = nc;
  for (int q = 0; q < std::min<int>(nc, cap); ++q) {
    if (rel_residual) rel_residual[q] = c->col_res[q];
    if (iterations) iterations[q] = c->col_its[q];
  }
  return HZ_OK;
}

int hz_krylov_basis(hz_ctx* c, double* V, int32_t cap, int32_t* nblocks, int32_t* ncols) {
  if (!c || !nblocks || !ncols || cap < 0 || (cap > 0 && !V)) return fail(HZ_EINVAL, "bad argument");
  if (c->s_cap == 0 || c->col_its.empty()) return fail(HZ_EINVAL, "no solve on this context yet");
  return guarded([&]() -> int {
    const int s = c->Kout.s;
    const int64_t n = c->space.n;
    int steps = 0;
    if (c->opt.block_arnoldi) {
      CK(cudaMemcpy(&steps, c->Bk.kb, sizeof(int), cudaMemcpyDeviceToHost));
    } else {
      std::vector<int> kc(s);
      CK(cudaMemcpy(kc.data(), c->Kout.kc, s * sizeof(int), cudaMemcpyDeviceToHost));
      for (int v : kc) steps = std::max(steps, v);
    }
    const int nb = std::min(steps + 1, c->opt.restart + 1);
    *nblocks = nb;
    *ncols = s;
    std::vector<double2> blk((size_t)n * s);
    for (int i = 0; i < std::min<int>(nb, cap); ++i) {
      CK(cudaMemcpy(blk.data(), (double2*)c->Kout.V + (size_t)i * n * s, blk.size() * sizeof(double2),
                    cudaMemcpyDeviceToHost));
      for (int q = 0; q < s; ++q)
        for (int64_t r = 0; r < n; ++r) {
          V[2 * (((size_t)i * s + q) * n + r)] = blk[r * s + q].x;
          V[2 * (((size_t)i * s + q) * n + r) + 1] = blk[r * s + q].y;
        }
    }
    return HZ_OK;
  });
}

int hz_profile_begin(hz_ctx* c) {
  if (!c) return fail(HZ_EINVAL, "NULL context");
  return guarded([&]() -> int {
    CK(cudaStreamSynchronize(c->st));
    c->prof.recs.clear();
    c->prof.used = 0;
    c->prof.on = true;
    return HZ_OK;
  });
}

int hz_profile_end(hz_ctx* c, hz_phase_time* out, int32_t cap, int32_t* count) {
  if (!c || !out || !count || cap < 0) return fail(HZ_EINVAL, "bad argument");
  return guarded([&]() -> int {
    CK(cudaStreamSynchronize(c->st));
    c->prof.on = false;
    hz_phase_time acc[PH_COUNT];
    for (int p = 0; p < PH_COUNT; ++p) acc[p] = hz_phase_time{PHASE_NAMES[p], 0, 0.0, 0.0, 0.0};
    for (auto& r : c->prof.recs) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, r.a, r.b));
      acc[r.ph].calls++;
      acc[r.ph].ms += ms;
      acc[r.ph].flops += r.flops;
      acc[r.ph].bytes += r.bytes;
    }
    c->prof.recs.clear();
    c->prof.used = 0;
    int nout = std::min<int>(cap, PH_COUNT);
    for (int p = 0; p < nout; ++p) out[p] = acc[p];
    *count = nout;
    return HZ_OK;
  });
}

int hz_matrix_csr(const hz_ctx* c, int64_t* rowptr, int32_t* col, double* val) {
  if (!c || !rowptr || !col || !val) return fail(HZ_EINVAL, "NULL argument");
  const CsrC& A = c->A_host;
  std::memcpy(rowptr, A.rowptr.data(), A.rowptr.size() * sizeof(int64_t));
  std::memcpy(col, A.col.data(), A.col.size() * sizeof(int32_t));
  for (size_t i = 0; i < A.val.size(); ++i) {
    val[2 * i] = A.val[i].real();
    val[2 * i + 1] = A.val[i].imag();
  }
  return HZ_OK;
}

// Copy an [s][n] complex block from the caller into c->B (rows layout).
static void load_block(hz_ctx* c, const double* F, int s, int on_device) {
  const int64_t n = c->space.n;
  const double2* src = reinterpret_cast<const double2*>(F);
  if (!on_device) {
    CK(cudaMemcpyAsync(c->U, F, (size_t)n * s * sizeof(double2), cudaMemcpyHostToDevice, c->st));
    src = c->U;
  }
  transpose_to_rows(src, c->B, n, s, c->st);
}

static void store_block(hz_ctx* c, const double2* Brow, double* out, int s, int on_device) {
  const int64_t n = c->space.n;
  double2* dst = on_device ? reinterpret_cast<double2*>(out) : c->U;
  transpose_from_rows(Brow, dst, n, s, c->st);
  if (!on_device) CK(cudaMemcpyAsync(out, c->U, (size_t)n * s * sizeof(double2), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
}

int hz_apply_A(hz_ctx* c, const double* X, double* Y, int32_t s, int32_t on_device) {
  if (!c || !X || !Y || s < 1 || s > c->opt.max_block) return fail(HZ_EINVAL, "bad argument");
  return guarded([&]() -> int {
    join_user(c);
    ensure_workspace(c, s);
    load_block(c, X, s, on_device);
    spmm_A(c, c->B, c->R, nullptr, s, 0);  // recorded in the "spmm_A" phase while profiling
    check_launch();
    store_block(c, c->R, Y, s, on_device);
    return HZ_OK;
  });
}

int hz_apply_prec(hz_ctx* c, const double* X, double* Y, int32_t s, int32_t on_device) {
  if (!c || !X || !Y || s < 1 || s > c->opt.max_block) return fail(HZ_EINVAL, "bad argument");
  return guarded([&]() -> int {
    join_user(c);
    ensure_workspace(c, s);
    load_block(c, X, s, on_device);
    apply_prec(c, c->B, c->R, s);
    check_launch();
    store_block(c, c->R, Y, s, on_device);
    check_sweep_flags(c);
    return HZ_OK;
  });
}

int hz_solve_rhs(hz_ctx* c, const double* F, int32_t ns, int32_t F_on_device, double* u, int32_t u_on_device,
                 hz_stats* stats) {
  if (!c || !F || !u || ns < 0) return fail(HZ_EINVAL, "bad argument");
  return guarded([&]() -> int {
    join_user(c);
    const double t0 = now_s();
    const int64_t n = c->space.n;
    c->col_res.clear();
    c->col_its.clear();
    int rc = HZ_OK;
    hz_stats agg;
    std::memset(&agg, 0, sizeof(agg));
    agg.converged = 1;
    for (int q0 = 0; q0 < ns; q0 += c->opt.max_block) {
      const int s = std::min(c->opt.max_block, ns - q0);
      ensure_workspace(c, s);
      load_block(c, F + 2 * (size_t)q0 * n, s, F_on_device);
      hz_stats st1;
      int r = fgmres(c, s, &st1);
      check_launch();
      store_block(c, c->X, u + 2 * (size_t)q0 * n, s, u_on_device);
      if (r != HZ_OK) rc = r;
      agg.iterations = std::max(agg.iterations, st1.iterations);
      agg.restarts += st1.restarts;
      agg.converged &= st1.converged;
      agg.max_rel_residual = std::max(agg.max_rel_residual, st1.max_rel_residual);
    }
    agg.ncols = ns;
    agg.solve_seconds = now_s() - t0;
    agg.setup_seconds = c->setup_s;
    agg.factor_seconds = c->factor_s;
    agg.perturbed_pivots = c->perturbed;
    check_sweep_flags(c);
    if (stats) *stats = agg;
    if (rc != HZ_OK) g_last_error = "FGMRES reached maxit before rtol";
    return rc;
  });
}

int hz_solve(hz_ctx* c, const double* src_xyz, const double* src_amp, int32_t ns, double* u, int32_t u_on_device,
             hz_stats* stats) {
  if (!c || !src_xyz || !src_amp || !u || ns < 0) return fail(HZ_EINVAL, "bad argument");
  return guarded([&]() -> int {
    join_user(c);
    const double t0 = now_s();
    const int64_t n = c->space.n;
    c->col_res.clear();
    c->col_its.clear();
    std::vector<int64_t> elem(ns);
    std::vector<double> lam(4 * (size_t)ns);
    locate_points(c->fine, src_xyz, ns, elem.data(), lam.data());
    for (int q = 0; q < ns; ++q)
      if (elem[q] < 0) throw HzError{HZ_EINVAL, "source outside the mesh"};
    int rc = HZ_OK;
    hz_stats agg;
    std::memset(&agg, 0, sizeof(agg));
    agg.converged = 1;
    for (int q0 = 0; q0 < ns; q0 += c->opt.max_block) {
      const int s = std::min(c->opt.max_block, ns - q0);
      ensure_workspace(c, s);
      std::vector<int> idx;
      std::vector<double2> val;
      for (int q = 0; q < s; ++q) {
        double phi[NLOC];
        p3_basis(&lam[4 * (q0 + q)], phi);
        const double ar = src_amp[2 * (q0 + q)], ai = src_amp[2 * (q0 + q) + 1];
        for (int i = 0; i < NLOC; ++i) {
          int64_t g = c->space.l2g[NLOC * elem[q0 + q] + i];
          if (c->space.dirichlet[g]) continue;
          idx.push_back((int)(g * s + q));
          val.push_back(make_double2(ar * phi[i], ai * phi[i]));
        }
      }
      if ((int)idx.size() > c->src_cap) {
        CK(cudaStreamSynchronize(c->st));
        if (c->d_srcidx) cudaFree(c->d_srcidx);
        if (c->d_srcval) cudaFree(c->d_srcval);
        c->d_srcidx = nullptr;
        c->d_srcval = nullptr;
        CK(cudaMalloc(&c->d_srcidx, idx.size() * sizeof(int)));
        CK(cudaMalloc(&c->d_srcval, val.size() * sizeof(double2)));
        c->src_cap = (int)idx.size();
      }
      CK(cudaMemcpyAsync(c->d_srcidx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice, c->st));
      CK(cudaMemcpyAsync(c->d_srcval, val.data(), val.size() * sizeof(double2), cudaMemcpyHostToDevice, c->st));
      axpy_cols_zero(c->B, n * s, c->st);
      scatter_point_sources(c->B, n, s, c->d_srcidx, c->d_srcval, (int)idx.size(), c->st);
      hz_stats st1;
      int r = fgmres(c, s, &st1);
      check_launch();
      store_block(c, c->X, u + 2 * (size_t)q0 * n, s, u_on_device);
      if (r != HZ_OK) rc = r;
      agg.iterations = std::max(agg.iterations, st1.iterations);
      agg.restarts += st1.restarts;
      agg.converged &= st1.converged;
      agg.max_rel_residual = std::max(agg.max_rel_residual, st1.max_rel_residual);
    }
    agg.ncols = ns;
    agg.solve_seconds = now_s() - t0;
    agg.setup_seconds = c->setup_s;
    agg.factor_seconds = c->factor_s;
    agg.perturbed_pivots = c->perturbed;
    check_sweep_flags(c);
    if (stats) *stats = agg;
    if (rc != HZ_OK) g_last_error = "FGMRES reached maxit before rtol";
    return rc;
  });
}

void hz_free(hz_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->st);
  c->work.release();
  c->pool.release();
  if (c->h_res) cudaFreeHost(c->h_res);
  if (c->h_done) cudaFreeHost(c->h_done);
  if (c->d_srcidx) cudaFree(c->d_srcidx);
  if (c->d_srcval) cudaFree(c->d_srcval);
  c->prof.destroy();
  c->g_fronts.reset();
  c->g_coarse.reset();
  for (DevMF* mf : {&c->lf.mf, &c->lc.mf}) destroy_side(*mf);
  cudaStreamDestroy(c->st);
  cudaEventDestroy(c->ev_join);
  delete c;
}

const char* hz_strerror(int code) {
  switch (code) {
    case HZ_OK: return "ok";
    case HZ_EINVAL: return "invalid argument";
    case HZ_ENOMEM: return "out of memory";
    case HZ_ECUDA: return "CUDA error";
    case HZ_EINTERNAL: return "internal error";
    case HZ_ESINGULAR: return "singular local matrix";
    case HZ_ENOTCONV: return "not converged";
    case HZ_EBREAKDOWN: return "Krylov breakdown";
    default: return "unknown error";
  }
}

const char* hz_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// Continuous batching of point-source requests (hz_server_*)
// ---------------------------------------------------------------------------
namespace {

// right-hand-side entries of one point source in column col of an [n][s] block
void point_source_entries(const hz_ctx* c, const double* xyz, const double* amp, int s, int col,
                          std::vector<int>& idx, std::vector<double2>& val) {
  int64_t e = -1;
  double lam[4];
  locate_points(c->fine, xyz, 1, &e, lam);
  if (e < 0) throw HzError{HZ_EINVAL, "source outside the mesh"};
  double phi[NLOC];
  p3_basis(lam, phi);
  for (int i = 0; i < NLOC; ++i) {
    const int64_t g = c->space.l2g[NLOC * e + i];
    if (c->space.dirichlet[g]) continue;
    idx.push_back((int)(g * s + col));
    val.push_back(make_double2(amp[0] * phi[i], amp[1] * phi[i]));
  }
}

void upload_sources(hz_ctx* c, const std::vector<int>& idx, const std::vector<double2>& val) {
  cudaStream_t st = c->st;
  if ((int)idx.size() > c->src_cap) {
    CK(cudaStreamSynchronize(st));
    if (c->d_srcidx) cudaFree(c->d_srcidx);
    if (c->d_srcval) cudaFree(c->d_srcval);
    c->d_srcidx = nullptr;
    c->d_srcval = nullptr;
    c->src_cap = 0;
    CK(cudaMalloc(&c->d_srcidx, idx.size() * sizeof(int)));
    CK(cudaMalloc(&c->d_srcval, val.size() * sizeof(double2)));
    c->src_cap = (int)idx.size();
  }
  CK(cudaMemcpyAsync(c->d_srcidx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(c->d_srcval, val.data(), val.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
}

}  // namespace

struct hz_server {
  hz_ctx* c = nullptr;
  int s = 0;
  struct Col {
    int64_t req;
    int idx;
  };
  struct Req {
    int ns = 0, remaining = 0, iterations = 0, converged = 1;
    double maxrel = 0.0;
    std::vector<double> xyz, amp;
    std::vector<double2> u;  // [ns][n] results
  };
  std::deque<Col> queue;
  std::vector<Col> slot;  // req = -1: free
  std::vector<int> slot_its;
  std::vector<double> slot_bn;
  std::map<int64_t, Req> reqs;
  std::deque<int64_t> finished;  // finished request ids not yet returned by hz_server_step
  // the slots' right-hand sides, iterates and residuals persist across
  // steps: the server owns them and lends them to the context for each step
  double2 *B = nullptr, *X = nullptr, *R = nullptr, *d_col = nullptr;
  ~hz_server() {
    if (c) cudaStreamSynchronize(c->st);
    for (double2* p : {B, X, R, d_col})
      if (p) cudaFree(p);
  }
  struct Lend {  // swaps the server's blocks into the context for one step
    hz_ctx* c;
    double2 *B, *X, *R;
    explicit Lend(hz_server* v) : c(v->c), B(v->c->B), X(v->c->X), R(v->c->R) {
      c->B = v->B;
      c->X = v->X;
      c->R = v->R;
    }
    ~Lend() {
      c->B = B;
      c->X = X;
      c->R = R;
    }
  };
};

// Device bytes that one right-hand-side column adds to a server on this
// context: the server's own B, X, R columns plus the context workspace of
// one column (the blocks of M^{-1} and of the outer Krylov basis, the local
// sub-vectors and front vectors of both levels, the inner coarse Krylov
// basis), as ensure_workspace allocates them.
static double column_bytes(const hz_ctx* c) {
  const double n = (double)c->space.n, m = c->opt.restart;
  const double ef = c->lf.mf.fp32 ? 8.0 : 16.0;
  double b = 3.0 * 16.0 * n;                                    // server B, X, R
  b += 6.0 * 16.0 * n;                                          // context B, X, R, T, Q, U
  b += ef * ((double)c->lf.sub_rows + (double)c->lf.mf.rows_total + (double)c->lf.mf.max_slots * MF_TILE_ROWS);
  b += 16.0 * n * (2.0 * m + 2.0);                              // V, Zk, W
  if (c->df) b += 16.0 * n * 2.0;                               // double-float W and product input
  if (c->has_coarse) {
    const double nh = (double)c->cspace.n, ec = c->lc.mf.fp32 ? 8.0 : 16.0, ek = c->coarse32 ? 8.0 : 16.0;
    const double mi = std::max(1, c->opt.coarse_inner_its);
    b += 2.0 * 16.0 * nh;                                       // r_H, y_H
    b += ec * ((double)c->lc.sub_rows + (double)c->lc.mf.rows_total + (double)c->lc.mf.max_slots * MF_TILE_ROWS);
    if (c->opt.coarse_mode == HZ_COARSE_GMRES) b += ek * nh * (2.0 * mi + 2.0);
    if (c->df && !c->coarse32 && c->opt.coarse_mode == HZ_COARSE_GMRES) b += 16.0 * nh * 2.0;
    if (c->coarse32) b += 8.0 * (2.0 * nh + 3.0 * n);
  }
  return b;
}

extern "C" int hz_server_column_bytes(const hz_ctx* c, double* bytes) {
  if (!c || !bytes) return fail(HZ_EINVAL, "bad argument");
  *bytes = column_bytes(c);
  return HZ_OK;
}

extern "C" int hz_server_create(hz_ctx* c, int32_t slots, hz_server** out) {
  if (!c || !out || slots < 1 || slots > c->opt.max_block) return fail(HZ_EINVAL, "bad argument");
  *out = nullptr;
  return guarded([&]() -> int {
    std::unique_ptr<hz_server> v(new hz_server());
    v->c = c;
    v->s = slots;
    join_user(c);
    ensure_workspace(c, slots);
    v->slot.assign(slots, hz_server::Col{-1, 0});
    v->slot_its.assign(slots, 0);
    v->slot_bn.assign(slots, 0.0);
    const int64_t vs = c->space.n * slots;
    for (double2** p : {&v->B, &v->X, &v->R}) {
      if (cudaMalloc(p, vs * sizeof(double2)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        throw HzError{HZ_ENOMEM, "server block allocation failed"};
      }
      axpy_cols_zero(*p, vs, c->st);
    }
    if (cudaMalloc(&v->d_col, c->space.n * sizeof(double2)) != cudaSuccess) {
      cudaGetLastError();
      v->d_col = nullptr;
      throw HzError{HZ_ENOMEM, "server column allocation failed"};
    }
    check_launch();
    CK(cudaStreamSynchronize(c->st));
    *out = v.release();
    return HZ_OK;
  });
}

extern "C" int hz_server_submit(hz_server* v, int64_t id, const double* src_xyz, const double* src_amp, int32_t ns) {
  if (!v || !src_xyz || !src_amp || ns < 1) return fail(HZ_EINVAL, "bad argument");
  if (v->reqs.count(id)) return fail(HZ_EINVAL, "request id already in use");
  return guarded([&]() -> int {
    hz_server::Req r;
    r.ns = r.remaining = ns;
    r.xyz.assign(src_xyz, src_xyz + 3 * (size_t)ns);
    r.amp.assign(src_amp, src_amp + 2 * (size_t)ns);
    std::vector<int64_t> elem(ns);
    std::vector<double> lam(4 * (size_t)ns);
    locate_points(v->c->fine, r.xyz.data(), ns, elem.data(), lam.data());
    for (int q = 0; q < ns; ++q)  // reject sources outside the mesh up front
      if (elem[q] < 0) throw HzError{HZ_EINVAL, "source outside the mesh"};
    v->reqs.emplace(id, std::move(r));
    for (int q = 0; q < ns; ++q) v->queue.push_back(hz_server::Col{id, q});
    return HZ_OK;
  });
}

extern "C" int hz_server_step(hz_server* v, int64_t* done_ids, int32_t cap, int32_t* ndone) {
  if (!v || !ndone || cap < 0 || (cap > 0 && !done_ids)) return fail(HZ_EINVAL, "bad argument");
  *ndone = 0;
  // hand out up to cap finished ids (oldest first); the rest wait for the next step
  auto drain = [&]() {
    while (*ndone < cap && !v->finished.empty()) {
      done_ids[(*ndone)++] = v->finished.front();
      v->finished.pop_front();
    }
  };
  return guarded([&]() -> int {
    hz_ctx* c = v->c;
    cudaStream_t st = c->st;
    const int s = v->s;
    const int64_t n = c->space.n;
    join_user(c);
    ensure_workspace(c, s);
    hz_server::Lend lend(v);
    // admit queued columns into free slots
    std::vector<int> idx;
    std::vector<double2> val;
    for (int q = 0; q < s && !v->queue.empty(); ++q) {
      if (v->slot[q].req >= 0) continue;
      const hz_server::Col col = v->queue.front();
      v->queue.pop_front();
      const hz_server::Req& r = v->reqs.at(col.req);
      v->slot[q] = col;
      v->slot_its[q] = 0;
      point_source_entries(c, &r.xyz[3 * (size_t)col.idx], &r.amp[2 * (size_t)col.idx], s, q, idx, val);
    }
    int active = 0;
    for (int q = 0; q < s; ++q) active += v->slot[q].req >= 0;
    if (active == 0) {
      drain();
      return HZ_OK;
    }
    if (!idx.empty()) {
      upload_sources(c, idx, val);
      scatter_point_sources(c->B, n, s, c->d_srcidx, c->d_srcval, (int)idx.size(), st);
      for (int q = 0; q < s; ++q)  // new columns start from X = 0, so R = B
        if (v->slot[q].req >= 0 && v->slot_its[q] == 0) col_copy(c->B, c->R, n, s, q, st);
    }
    // per-slot tolerances (free slots: 0; their zero residual counts as done)
    column_norms(c->B, n, s, c->bnorm, c->Kout, st);
    CK(cudaMemcpyAsync(c->h_res, c->bnorm, s * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    std::vector<double> tol(s);
    for (int q = 0; q < s; ++q) {
      v->slot_bn[q] = c->h_res[q];
      tol[q] = v->slot[q].req >= 0 ? c->opt.rtol * v->slot_bn[q] : 0.0;
    }
    CK(cudaMemcpyAsync(c->Kout.tol, tol.data(), s * sizeof(double), cudaMemcpyHostToDevice, st));
    // one restart cycle for every slot, then the true residuals
    int maxleft = 1;
    for (int q = 0; q < s; ++q)
      if (v->slot[q].req >= 0) maxleft = std::max(maxleft, c->opt.maxit - v->slot_its[q]);
    fgmres_cycle(c, s, std::min(c->opt.restart, maxleft));
    std::vector<int> kc(s);  // Arnoldi steps each column accepted in this cycle
    CK(cudaMemcpyAsync(kc.data(), c->Kout.kc, s * sizeof(int), cudaMemcpyDeviceToHost, st));
    true_residual(c, s);
    check_launch();
    for (int q = 0; q < s; ++q) {
      if (v->slot[q].req < 0) continue;
      v->slot_its[q] += std::max(kc[q], 1);  // at least one: a stalled column still reaches maxit
      const double rel = v->slot_bn[q] > 0 ? c->h_res[q] / v->slot_bn[q] : 0.0;
      const bool conv = rel <= c->opt.rtol;
      if (!conv && v->slot_its[q] < c->opt.maxit) continue;
      hz_server::Req& r = v->reqs.at(v->slot[q].req);
      if (r.u.empty()) r.u.resize((size_t)r.ns * n);
      col_get(c->X, v->d_col, n, s, q, st);
      CK(cudaMemcpyAsync(&r.u[(size_t)v->slot[q].idx * n], v->d_col, n * sizeof(double2), cudaMemcpyDeviceToHost,
                         st));
      CK(cudaStreamSynchronize(st));  // d_col is reused by the next retired slot
      r.iterations = std::max(r.iterations, v->slot_its[q]);
      r.converged &= conv ? 1 : 0;
      r.maxrel = std::max(r.maxrel, rel);
      col_zero(c->B, n, s, q, st);
      col_zero(c->X, n, s, q, st);
      col_zero(c->R, n, s, q, st);
      if (--r.remaining == 0) v->finished.push_back(v->slot[q].req);
      v->slot[q].req = -1;
    }
    check_launch();
    CK(cudaStreamSynchronize(st));
    check_sweep_flags(c);
    drain();
    return HZ_OK;
  });
}

extern "C" int hz_server_fetch(hz_server* v, int64_t id, double* u, hz_stats* stats) {
  if (!v || !u) return fail(HZ_EINVAL, "bad argument");
  auto it = v->reqs.find(id);
  if (it == v->reqs.end() || it->second.remaining != 0) return fail(HZ_EINVAL, "request unknown or not finished");
  hz_server::Req& r = it->second;
  std::memcpy(u, r.u.data(), r.u.size() * sizeof(double2));
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->iterations = r.iterations;
    stats->converged = r.converged;
    stats->ncols = r.ns;
    stats->max_rel_residual = r.maxrel;
  }
  const int rc = r.converged ? HZ_OK : HZ_ENOTCONV;
  if (rc != HZ_OK) g_last_error = "FGMRES reached maxit before rtol";
  v->reqs.erase(it);
  return rc;
}

extern "C" int hz_server_pending(const hz_server* v, int32_t* queued, int32_t* active) {
  if (!v || !queued || !active) return fail(HZ_EINVAL, "bad argument");
  *queued = (int32_t)v->queue.size();
  int a = 0;
  for (const auto& q : v->slot) a += q.req >= 0;
  *active = a;
  return HZ_OK;
}

extern "C" void hz_server_free(hz_server* v) { delete v; }

// ---------------------------------------------------------------------------
// FWI misfit and adjoint-state gradient (hz_receiver_operator, hz_fwi_gradient)
// ---------------------------------------------------------------------------
namespace {

struct TmpPool {  // device buffers of one call, released after the stream drains
  DevPool p;
  cudaStream_t st;
  ~TmpPool() {
    cudaStreamSynchronize(st);
    p.release();
  }
};

void fwi_prepare(hz_ctx* c) {
  if (c->fwi_ready) return;
  const Mesh& m = c->fine;
  const int64_t ne = m.ne;
  std::vector<int> l2g((size_t)ne * NLOC);
  std::vector<double> vol(ne), farea((size_t)ne * 4, 0.0);
  for (int64_t e = 0; e < ne; ++e) {
    double P[12];
    for (int a = 0; a < 4; ++a)
      for (int d = 0; d < 3; ++d) P[3 * a + d] = m.xyz[3 * m.tets[4 * e + a] + d];
    vol[e] = elem_geom(P).vol;
    for (int f = 0; f < 4; ++f)
      if (m.nbr[4 * e + f] < 0 && m.ftag[4 * e + f] == HZ_BC_ROBIN) farea[4 * e + f] = face_area(P, f);
    for (int i = 0; i < NLOC; ++i) {
      const int64_t g = c->space.l2g[NLOC * e + i];
      l2g[NLOC * e + i] = c->space.dirichlet[g] ? -1 : (int)g;
    }
  }
  c->d_fwi_l2g = c->pool.upload(l2g, c->st);
  c->d_fwi_vol = c->pool.upload(vol, c->st);
  c->d_fwi_farea = c->pool.upload(farea, c->st);
  c->d_fwi_m = c->pool.upload(c->mvals, c->st);
  CK(cudaStreamSynchronize(c->st));
  c->fwi_ready = true;
}

void receiver_operator(const hz_ctx* c, const double* rec_xyz, int nr, int32_t* idx, double* w) {
  std::vector<int64_t> elem(nr);
  std::vector<double> lam(4 * (size_t)nr);
  locate_points(c->fine, rec_xyz, nr, elem.data(), lam.data());
  for (int k = 0; k < nr; ++k) {
    if (elem[k] < 0) throw HzError{HZ_EINVAL, "receiver outside the mesh"};
    double phi[NLOC];
    p3_basis(&lam[4 * (size_t)k], phi);
    for (int i = 0; i < NLOC; ++i) {
      const int64_t g = c->space.l2g[NLOC * elem[k] + i];
      const bool keep = !c->space.dirichlet[g] && phi[i] != 0.0;
      idx[(size_t)k * NLOC + i] = keep ? (int32_t)g : -1;
      w[(size_t)k * NLOC + i] = keep ? phi[i] : 0.0;
    }
  }
}

}  // namespace

extern "C" int hz_receiver_operator(const hz_ctx* c, const double* rec_xyz, int32_t nr, int32_t* idx, double* w) {
  if (!c || nr < 0 || (nr > 0 && (!rec_xyz || !idx || !w))) return fail(HZ_EINVAL, "bad argument");
  return guarded([&]() -> int {
    receiver_operator(c, rec_xyz, nr, idx, w);
    return HZ_OK;
  });
}

extern "C" int hz_fwi_gradient(hz_ctx* c, const double* src_xyz, const double* src_amp, int32_t ns,
                               const double* rec_xyz, int32_t nr, const double* d_obs, double* chi, double* grad,
                               double* d_syn, hz_stats* stats) {
  if (!c || !src_xyz || !src_amp || !rec_xyz || !grad || ns < 1 || nr < 1) return fail(HZ_EINVAL, "bad argument");
  return guarded([&]() -> int {
    join_user(c);
    const double t0 = now_s();
    const int64_t n = c->space.n, ne = c->fine.ne;
    c->col_res.clear();
    c->col_its.clear();
    std::vector<double> fwd_res, adj_res;
    std::vector<int> fwd_its, adj_its;
    cudaStream_t st = c->st;
    // receivers: P as [nr][20] (dof, weight) and its transpose in CSR over the touched dofs
    std::vector<int> pidx((size_t)nr * NLOC);
    std::vector<double> pw((size_t)nr * NLOC);
    receiver_operator(c, rec_xyz, nr, pidx.data(), pw.data());
    std::map<int, std::vector<std::pair<int, double>>> rows;
    for (int k = 0; k < nr; ++k)
      for (int i = 0; i < NLOC; ++i)
        if (pidx[(size_t)k * NLOC + i] >= 0) rows[pidx[(size_t)k * NLOC + i]].push_back({k, pw[(size_t)k * NLOC + i]});
    std::vector<int> trow, tptr{0}, tk;
    std::vector<double> tw;
    for (auto& kv : rows) {
      trow.push_back(kv.first);
      for (auto& e : kv.second) {
        tk.push_back(e.first);
        tw.push_back(e.second);
      }
      tptr.push_back((int)tk.size());
    }
    const int nt = (int)trow.size();
    fwi_prepare(c);
    const P3Tables& T = p3_tables();
    CK(fwi_set_tables(&T.M[0][0], &T.B[0][0][0], st));
    TmpPool tmp{DevPool(), st};
    int* d_pidx = tmp.p.upload(pidx, st);
    double* d_pw = tmp.p.upload(pw, st);
    int* d_trow = tmp.p.upload(trow, st);
    int* d_tptr = tmp.p.upload(tptr, st);
    int* d_tk = tmp.p.upload(tk, st);
    double* d_tw = tmp.p.upload(tw, st);
    double* d_g = tmp.p.alloc<double>(ne);
    double* d_chi = tmp.p.alloc<double>(1);
    const int bs = std::min<int>(c->opt.max_block, ns);
    double2* d_r = tmp.p.alloc<double2>((size_t)bs * nr);
    double2* d_d = tmp.p.alloc<double2>((size_t)bs * nr);
    double2* d_u = tmp.p.alloc<double2>((size_t)n * bs);
    CK(cudaMemsetAsync(d_g, 0, ne * sizeof(double), st));
    CK(cudaMemsetAsync(d_chi, 0, sizeof(double), st));
    int rc = HZ_OK;
    hz_stats agg;
    std::memset(&agg, 0, sizeof(agg));
    agg.converged = 1;
    auto add_stats = [&](const hz_stats& a) {
      agg.iterations = std::max(agg.iterations, a.iterations);
      agg.restarts += a.restarts;
      agg.converged &= a.converged;
      agg.max_rel_residual = std::max(agg.max_rel_residual, a.max_rel_residual);
    };
    std::vector<double2> h_r;
    for (int q0 = 0; q0 < ns; q0 += c->opt.max_block) {
      const int s = std::min(c->opt.max_block, ns - q0);
      ensure_workspace(c, s);
      // forward: A u = F (point sources)
      std::vector<int> idx;
      std::vector<double2> val;
      for (int q = 0; q < s; ++q)
        point_source_entries(c, &src_xyz[3 * (size_t)(q0 + q)], &src_amp[2 * (size_t)(q0 + q)], s, q, idx, val);
      int* d_si = tmp.p.upload(idx, st);
      double2* d_sv = tmp.p.upload(val, st);
      axpy_cols_zero(c->B, n * s, st);
      scatter_point_sources(c->B, n, s, d_si, d_sv, (int)idx.size(), st);
      hz_stats a;
      int r = fgmres(c, s, &a);
      check_launch();
      if (r != HZ_OK) rc = r;
      add_stats(a);
      // fgmres appended this block's columns: keep forward and adjoint columns apart
      fwd_res.insert(fwd_res.end(), c->col_res.end() - s, c->col_res.end());
      fwd_its.insert(fwd_its.end(), c->col_its.end() - s, c->col_its.end());
      CK(cudaMemcpyAsync(d_u, c->X, (size_t)n * s * sizeof(double2), cudaMemcpyDeviceToDevice, st));
      // residual at the receivers and misfit
      if (d_obs)
        CK(cudaMemcpyAsync(d_d, d_obs + 2 * (size_t)q0 * nr, (size_t)s * nr * sizeof(double2),
                           cudaMemcpyHostToDevice, st));
      fwi_residual(nr, s, d_pidx, d_pw, d_u, d_obs ? d_d : nullptr, d_r, st);
      fwi_chi((int64_t)s * nr, d_r, d_chi, st);
      if (d_syn) {
        h_r.resize((size_t)s * nr);
        CK(cudaMemcpyAsync(h_r.data(), d_r, h_r.size() * sizeof(double2), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (size_t i = 0; i < h_r.size(); ++i) {
          const double* dd = d_obs ? d_obs + 2 * ((size_t)q0 * nr + i) : nullptr;
          d_syn[2 * ((size_t)q0 * nr + i)] = h_r[i].x + (dd ? dd[0] : 0.0);
          d_syn[2 * ((size_t)q0 * nr + i) + 1] = h_r[i].y + (dd ? dd[1] : 0.0);
        }
      }
      // adjoint: A lambda = P^T conj(r)
      axpy_cols_zero(c->B, n * s, st);
      fwi_adjoint_rhs(nt, s, nr, d_trow, d_tptr, d_tk, d_tw, d_r, c->B, st);
      r = fgmres(c, s, &a);
      check_launch();
      if (r != HZ_OK) rc = r;
      add_stats(a);
      adj_res.insert(adj_res.end(), c->col_res.end() - s, c->col_res.end());
      adj_its.insert(adj_its.end(), c->col_its.end() - s, c->col_its.end());
      // g_e -= Re sum_s lambda_e^T dA/dm_e u_e
      fwi_gradient(ne, s, c->d_fwi_l2g, c->d_fwi_vol, c->d_fwi_farea, c->d_fwi_m, c->omega, d_u, c->X, d_g, st);
      check_launch();
    }
    CK(cudaMemcpyAsync(grad, d_g, ne * sizeof(double), cudaMemcpyDeviceToHost, st));
    double h_chi = 0;
    CK(cudaMemcpyAsync(&h_chi, d_chi, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (chi) *chi = h_chi;
    c->col_res = fwd_res;
    c->col_res.insert(c->col_res.end(), adj_res.begin(), adj_res.end());
    c->col_its = fwd_its;
    c->col_its.insert(c->col_its.end(), adj_its.begin(), adj_its.end());
    agg.ncols = 2 * ns;
    agg.solve_seconds = now_s() - t0;
    agg.setup_seconds = c->setup_s;
    agg.factor_seconds = c->factor_s;
    agg.perturbed_pivots = c->perturbed;
    check_sweep_flags(c);
    if (stats) *stats = agg;
    if (rc != HZ_OK) g_last_error = "FGMRES reached maxit before rtol";
    return rc;
  });
}
