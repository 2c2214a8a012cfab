// oz_grouped.cu -- many products in one launch per phase (oz_group_create /
// oz_group_run): the five phases of Sec. "Structure" run over all products
// of a plan at once, the split of every A, then of every B, the GEMMs of
// every product as one persistent kernel, and one reconstruct. A block of a
// split or reconstruct launch finds its product in a block map (one int per
// block, per phase); a GEMM CTA finds the product of its first unit by a binary
// search over the products' first unit indices and walks forward from there.
// Both the product table and the maps are device memory written once, at
// create time.
//
// Products of different tables form separate groups, and the groups run side
// by side on streams the group object owns (forked from and joined back to
// the caller's stream, so a run can be captured into a CUDA graph); within a
// group the splits of A and of B run side by side too. The groups' GEMMs run
// one after another, on CTA pairs or one CTA per tile (group_uses_pairs).
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "oz_internal.h"

namespace {

using oz::round_up;

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// A group's GEMMs run on CTA pairs (256 x 256 tiles: a third less shared-memory
// traffic per product than one CTA per 128 x 256 tile) when its units hold at
// least one 1024-term slab on average; groups of shorter products run one CTA
// per 128 x 256 tile, which pads fewer rows (their units are bound by the
// epilogue, not by the products). Measured on the 256-product batch: the
// k > 836 set 6.14 ms with pairs against 6.39 ms, the k <= 836 set 3.50 ms
// against 2.86 ms.
bool group_uses_pairs(const std::vector<int>& mem, const int64_t* mnk) {
  double units = 0, kb = 0;
  for (int i : mem) {
    const int64_t m = mnk[3 * i], n = mnk[3 * i + 1], k = mnk[3 * i + 2];
    const double u = (double)((m + 255) / 256) * ((n + 255) / 256);
    units += u;
    kb += u * (double)(round_up(k, oz::kPadK) / 64);
  }
  return units > 0 && kb >= 16.0 * units;
}

struct Group {
  oz_plan plan;
  int first, count;                     // range of the device table
  int64_t total_rows, total_wrows, total_cm, total_sh, total_sc, total_units, total_rec;
  bool pairs;                           // GEMMs on CTA pairs (else one CTA per tile)
  bool one_slab;                        // every product's k_pad at most 1024 (one slab per unit)
  oz::GroupMaps maps;                   // block -> problem (index from `first`) per phase
};

// threads per row chunk of the grouped reconstruct: the least power of two
// covering n / ept entries (ept entries per thread), within [8, 32]: chunks
// of at most 32 ept entries waste little of a row whose length is not a power
// of two (90 % of the threads busy on the 256-product batch, against 72 % with
// chunks up to 256 ept), and a block covers 256 / tpr rows
int rec_tpr(int64_t n, int ept) {
  int tpr = 8;
  while (tpr < 32 && ept * (int64_t)tpr < n) tpr *= 2;
  return tpr;
}

// Byte sizes of one product's part of the workspace (TC engine planes).
struct Part {
  int64_t m_pad, n_pad, k_pad, ldy;
  size_t s, t, u, v, y, total;
};

Part part_of(const oz_plan p, int64_t m, int64_t n, int64_t k) {
  Part P;
  P.m_pad = round_up(m > 0 ? m : 1, oz::kPadRows);
  P.n_pad = round_up(n > 0 ? n : 1, oz::kPadRows);
  P.k_pad = round_up(k > 0 ? k : 1, oz::kPadK);
  P.ldy = round_up(n > 0 ? n : 1, 16);
  size_t off = 0;
  P.s = off; off = al256(off + 4 * (size_t)m);
  P.t = off; off = al256(off + 4 * (size_t)n);
  P.u = off; off = al256(off + (size_t)p->Q * P.m_pad * P.k_pad * 2);
  P.v = off; off = al256(off + (size_t)p->Q * P.n_pad * P.k_pad * 2);
  P.y = off; off = al256(off + (size_t)p->Q * m * P.ldy);
  P.total = off;
  return P;
}

// entries per thread of the grouped reconstruct for a plan's products
int rec_ept(const oz_plan p) { return oz::reconstruct_grouped_eight(p->tab) ? 8 : 4; }

// Blocks of one product in each phase's launch.
struct Blocks {
  int64_t rows, wrows, cm, sh, sc, rec;
  int64_t total() const { return rows + wrows + cm + sh + sc + rec; }
};

Blocks blocks_of(const Part& P, int64_t m, int64_t n, int64_t k, int ept) {
  Blocks b;
  // one block per row, else one warp per row (eight rows per block: fewer,
  // fuller blocks on the short and middling rows of a batch)
  const bool long_rows = P.k_pad > 4096;
  b.rows = long_rows ? P.m_pad : 0;
  b.wrows = long_rows ? 0 : P.m_pad / 8;
  b.cm = ((n + 31) / 32) * ((k + 255) / 256);
  b.sh = (n + 255) / 256;
  b.sc = (P.n_pad / 32) * (P.k_pad / 64);
  const int tpr = rec_tpr(n, ept);
  b.rec = ((m + 256 / tpr - 1) / (256 / tpr)) * ((n + ept * (int64_t)tpr - 1) / (ept * (int64_t)tpr));
  return b;
}

// Plans with the same moduli and bit budget have the same tables: their
// products can share every launch.
bool same_tables(const oz_plan a, const oz_plan b) {
  if (a == b) return true;
  if (a->tab.Q != b->tab.Q || a->tab.bits != b->tab.bits) return false;
  for (int q = 0; q < a->tab.Q; ++q)
    if (a->tab.m[q] != b->tab.m[q]) return false;
  return true;
}

bool plan_ok(const oz_plan p) {
  return p && !p->is_fp && oz::engine_bf16(p->engine) && p->tab.limbs <= 4 && p->tab.npairs >= 5 &&
         p->tab.npairs <= 8 && p->tab.bits <= 64;
}

// Layout of the whole workspace: status word, table, block maps, column
// maxima, parts.
struct Layout {
  size_t table, maps, colmax, parts, total;
  std::vector<size_t> part_off;         // per caller index (0 for skipped products)
  std::vector<size_t> colmax_off;
};

bool layout(int count, const oz_plan* plans, const int64_t* mnk, Layout* L) {
  if (count < 0 || (count > 0 && (!plans || !mnk))) return false;
  size_t off = 256;                                       // status word (oz_query_status reads it)
  L->table = off;
  off = al256(off + sizeof(OzGroupProblem) * (size_t)(count > 0 ? count : 1));
  L->maps = off;
  for (int i = 0; i < count; ++i) {
    const int64_t m = mnk[3 * i], n = mnk[3 * i + 1], k = mnk[3 * i + 2];
    if (m < 0 || n < 0 || k < 0 || !plan_ok(plans[i])) return false;
    if (m == 0 || n == 0 || k == 0) continue;
    off += sizeof(int32_t) * (size_t)blocks_of(part_of(plans[i], m, n, k), m, n, k, rec_ept(plans[i])).total();
  }
  off = al256(off);
  L->colmax = off;
  L->colmax_off.assign(count, 0);
  for (int i = 0; i < count; ++i) {
    const int64_t n = mnk[3 * i + 1];
    if (n < 0) return false;
    L->colmax_off[i] = off;
    off += 8 * (size_t)n;
  }
  off = al256(off);
  L->parts = off;
  L->part_off.assign(count, 0);
  for (int i = 0; i < count; ++i) {
    const int64_t m = mnk[3 * i], n = mnk[3 * i + 1], k = mnk[3 * i + 2];
    if (m < 0 || n < 0 || k < 0 || !plan_ok(plans[i])) return false;
    if (m == 0 || n == 0 || k == 0) continue;
    L->part_off[i] = off;
    off += part_of(plans[i], m, n, k).total;
  }
  L->total = off;
  return true;
}

}  // namespace

struct oz_group_s {
  char* ws;
  size_t table_off, maps_off, colmax_off, colmax_bytes;
  std::vector<Group> groups;
  // products with k == 0: C = 0
  std::vector<double*> zero_c;
  std::vector<int64_t> zero_m, zero_n, zero_ldc;
  // per group: a stream for the A side (then GEMMs and reconstruct) and one
  // for the B side; events: fork, per group the B side done, the group done
  // and its GEMMs done
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  ~oz_group_s() {
    for (cudaEvent_t e : events) cudaEventDestroy(e);
    for (cudaStream_t st : streams) cudaStreamDestroy(st);
  }
};

extern "C" size_t oz_grouped_workspace_bytes(int count, const oz_plan* plans, const int64_t* mnk) {
  Layout L;
  if (!layout(count, plans, mnk, &L)) return 0;
  return L.total;
}

extern "C" oz_status oz_group_create(oz_group* out, int count, const oz_plan* plans, const int64_t* mnk,
                                     const double* const* A, const int64_t* lda, const double* const* B,
                                     const int64_t* ldb, double* const* C, const int64_t* ldc, void* workspace,
                                     size_t workspace_bytes) {
  if (!out) return OZ_ERR_INVALID_ARG;
  *out = nullptr;
  if (count < 0 || (count > 0 && (!plans || !mnk || !A || !B || !C || !lda || !ldb || !ldc)))
    return OZ_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i)
    if (!plans[i]) return OZ_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i)
    if (!plan_ok(plans[i])) return OZ_ERR_UNSUPPORTED;
  Layout L;
  if (!layout(count, plans, mnk, &L)) return OZ_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    const int64_t m = mnk[3 * i], n = mnk[3 * i + 1], k = mnk[3 * i + 2];
    if (lda[i] < (k > 1 ? k : 1) || ldb[i] < (n > 1 ? n : 1) || ldc[i] < (n > 1 ? n : 1)) return OZ_ERR_INVALID_ARG;
    if (k > plans[i]->k_max) return OZ_ERR_K_TOO_LARGE;
    if (m > 0 && n > 0 && (!C[i] || (reinterpret_cast<uintptr_t>(C[i]) & 7))) return OZ_ERR_INVALID_ARG;
    if (m > 0 && n > 0 && k > 0 &&
        (!A[i] || !B[i] || (reinterpret_cast<uintptr_t>(A[i]) & 7) || (reinterpret_cast<uintptr_t>(B[i]) & 7)))
      return OZ_ERR_INVALID_ARG;
  }
  if (!workspace || workspace_bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return OZ_ERR_WORKSPACE;

  oz_group g = new (std::nothrow) oz_group_s;
  if (!g) return OZ_ERR_INVALID_ARG;
  g->ws = static_cast<char*>(workspace);
  g->table_off = L.table;
  g->maps_off = L.maps;
  g->colmax_off = L.colmax;
  g->colmax_bytes = L.parts - L.colmax;

  // groups by tables (order of first appearance); within a group, longest k first
  std::vector<oz_plan> distinct;
  std::vector<std::vector<int>> members;
  for (int i = 0; i < count; ++i) {
    const int64_t m = mnk[3 * i], n = mnk[3 * i + 1], k = mnk[3 * i + 2];
    if (m == 0 || n == 0) continue;
    if (k == 0) {
      g->zero_c.push_back(C[i]);
      g->zero_m.push_back(m);
      g->zero_n.push_back(n);
      g->zero_ldc.push_back(ldc[i]);
      continue;
    }
    size_t gi = 0;
    while (gi < distinct.size() && !same_tables(distinct[gi], plans[i])) ++gi;
    if (gi == distinct.size()) {
      distinct.push_back(plans[i]);
      members.emplace_back();
    }
    members[gi].push_back(i);
  }
  std::vector<OzGroupProblem> table;
  std::vector<int32_t> maps;              // every group's block maps, phase after phase
  int32_t* status = reinterpret_cast<int32_t*>(g->ws);
  for (size_t gi = 0; gi < distinct.size(); ++gi) {
    std::vector<int>& mem = members[gi];
    std::stable_sort(mem.begin(), mem.end(), [&](int x, int y) { return mnk[3 * x + 2] > mnk[3 * y + 2]; });
    const oz_plan p = distinct[gi];
    Group G = {};
    G.plan = p;
    G.first = (int)table.size();
    G.count = (int)mem.size();
    G.pairs = group_uses_pairs(mem, mnk);
    G.one_slab = true;
    for (int i : mem) G.one_slab = G.one_slab && round_up(mnk[3 * i + 2], oz::kPadK) <= 1024;
    for (int i : mem) {
      const int64_t m = mnk[3 * i], n = mnk[3 * i + 1], k = mnk[3 * i + 2];
      const Part P = part_of(p, m, n, k);
      const Blocks nb = blocks_of(P, m, n, k, rec_ept(p));
      char* base = g->ws + L.part_off[i];
      OzGroupProblem pr;
      memset(&pr, 0, sizeof pr);
      pr.A = A[i];
      pr.B = B[i];
      pr.C = C[i];
      pr.lda = lda[i];
      pr.ldb = ldb[i];
      pr.ldc = ldc[i];
      pr.m = m;
      pr.n = n;
      pr.k = k;
      pr.m_pad = P.m_pad;
      pr.n_pad = P.n_pad;
      pr.k_pad = P.k_pad;
      pr.ldy = P.ldy;
      pr.U = base + P.u;
      pr.V = base + P.v;
      pr.Y = reinterpret_cast<uint8_t*>(base + P.y);
      pr.s = reinterpret_cast<int32_t*>(base + P.s);
      pr.t = reinterpret_cast<int32_t*>(base + P.t);
      pr.colmax = reinterpret_cast<uint64_t*>(g->ws + L.colmax_off[i]);
      pr.flag = status;
      pr.tiles_m = (int)((m + oz::kTileM - 1) / oz::kTileM);   // one-CTA tiles (pairs: ceil(m / 256))
      pr.tiles_n = (int)((n + 255) / 256);
      pr.kblocks = (int)(P.k_pad / 64);
      if (nb.rows > 0) {                // one block per row (the long products come first)
        pr.rows_begin = G.total_rows;
        G.total_rows += nb.rows;
      } else {                          // one warp per row, eight rows per block
        pr.rows_begin = G.total_wrows;
        G.total_wrows += nb.wrows;
      }
      pr.cm_begin = G.total_cm;
      G.total_cm += nb.cm;
      pr.sh_begin = G.total_sh;
      G.total_sh += nb.sh;
      pr.sc_begin = G.total_sc;
      G.total_sc += nb.sc;
      pr.unit_begin = G.total_units;
      G.total_units += (int64_t)p->Q * (G.pairs ? (m + 255) / 256 : pr.tiles_m) * pr.tiles_n;
      pr.rec_tpr = rec_tpr(n, rec_ept(p));
      pr.rec_begin = G.total_rec;
      G.total_rec += nb.rec;
      if (!oz::group_maps_tc(&pr, p->Q, G.pairs)) {
        delete g;
        return OZ_ERR_INVALID_ARG;
      }
      table.push_back(pr);
    }
    // block maps of the group: per phase, the index (from G.first) of the
    // problem of each block, in the order the begin fields were assigned
    auto append = [&](int64_t Blocks::*field) {
      const size_t at = maps.size();
      for (int li = 0; li < G.count; ++li) {
        const int i = mem[li];
        const int64_t m = mnk[3 * i], n = mnk[3 * i + 1], k = mnk[3 * i + 2];
        maps.insert(maps.end(), (size_t)(blocks_of(part_of(p, m, n, k), m, n, k, rec_ept(p)).*field), (int32_t)li);
      }
      return at;
    };
    const size_t at_rows = append(&Blocks::rows), at_wrows = append(&Blocks::wrows), at_cm = append(&Blocks::cm),
                 at_sh = append(&Blocks::sh), at_sc = append(&Blocks::sc), at_rec = append(&Blocks::rec);
    const int32_t* mb = reinterpret_cast<const int32_t*>(g->ws + L.maps);
    G.maps = {mb + at_rows, mb + at_wrows, mb + at_cm, mb + at_sh, mb + at_sc, mb + at_rec};
    g->groups.push_back(G);
  }
  if ((!table.empty() &&
       cudaMemcpy(g->ws + L.table, table.data(), sizeof(OzGroupProblem) * table.size(), cudaMemcpyHostToDevice) !=
           cudaSuccess) ||
      (!maps.empty() &&
       cudaMemcpy(g->ws + L.maps, maps.data(), sizeof(int32_t) * maps.size(), cudaMemcpyHostToDevice) != cudaSuccess)) {
    cudaGetLastError();
    delete g;
    return OZ_ERR_CUDA;
  }
  const size_t ng = g->groups.size();
  for (size_t i = 0; i < 2 * ng; ++i) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete g;
      return OZ_ERR_CUDA;
    }
    g->streams.push_back(st);
  }
  for (size_t i = 0; i < 1 + 3 * ng; ++i) {
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      delete g;
      return OZ_ERR_CUDA;
    }
    g->events.push_back(ev);
  }
  *out = g;
  return OZ_OK;
}

extern "C" oz_status oz_group_run(oz_group g, void* stream) {
  if (!g) return OZ_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the status word, and the column maxima of every B (atomicMax targets), start from zero
  cudaError_t e = cudaMemsetAsync(g->ws, 0, 16, st);
  if (e == cudaSuccess && g->colmax_bytes) e = cudaMemsetAsync(g->ws + g->colmax_off, 0, g->colmax_bytes, st);
  if (e != cudaSuccess) return OZ_ERR_CUDA;
  const OzGroupProblem* table = reinterpret_cast<const OzGroupProblem*>(g->ws + g->table_off);
  for (size_t i = 0; i < g->zero_c.size(); ++i) {
    e = cudaMemset2DAsync(g->zero_c[i], (size_t)g->zero_ldc[i] * 8, 0, (size_t)g->zero_n[i] * 8,
                          (size_t)g->zero_m[i], st);
    if (e != cudaSuccess) return OZ_ERR_CUDA;
  }
  int32_t* status = reinterpret_cast<int32_t*>(g->ws);
  cudaEvent_t fork = g->events[0];
  auto chk = [&](cudaError_t r) { if (e == cudaSuccess && r != cudaSuccess) e = r; };
  chk(cudaEventRecord(fork, st));
  for (size_t gi = 0; gi < g->groups.size(); ++gi) {
    const Group& G = g->groups[gi];
    const OzTables& T = G.plan->tab;
    const OzGroupProblem* probs = table + G.first;
    cudaStream_t sa = g->streams[2 * gi], sb = g->streams[2 * gi + 1];
    cudaEvent_t b_done = g->events[1 + 3 * gi], done = g->events[2 + 3 * gi], gemm_done = g->events[3 + 3 * gi];
    chk(cudaStreamWaitEvent(sa, fork, 0));
    chk(cudaStreamWaitEvent(sb, fork, 0));
    if (e == cudaSuccess) e = oz::launch_split_rows_grouped(T, probs, G.maps, G.total_rows, G.total_wrows, sa);
    if (e == cudaSuccess) e = oz::launch_split_cols_grouped(T, probs, G.maps, G.total_cm, G.total_sh, G.total_sc, sb);
    chk(cudaEventRecord(b_done, sb));
    chk(cudaStreamWaitEvent(sa, b_done, 0));
    // the groups' GEMMs run one after another: each fills every SM (a pair's
    // CTA all of its shared memory), so little is lost, and no two
    // tensor-memory users of this call run at once
    if (gi > 0) chk(cudaStreamWaitEvent(sa, g->events[3 + 3 * (gi - 1)], 0));
    if (e == cudaSuccess) e = oz::launch_gemm_tc_grouped(T, probs, G.count, G.total_units, status, sa, G.pairs, G.one_slab);
    chk(cudaEventRecord(gemm_done, sa));
    if (e == cudaSuccess) e = oz::launch_reconstruct_grouped(T, probs, G.maps, G.total_rec, sa);
    chk(cudaEventRecord(done, sa));
    chk(cudaStreamWaitEvent(st, done, 0));
  }
  return e == cudaSuccess ? OZ_OK : OZ_ERR_CUDA;
}

extern "C" void oz_group_destroy(oz_group g) { delete g; }
