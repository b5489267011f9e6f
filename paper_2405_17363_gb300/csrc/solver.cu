// Host layer of the C ABI (include/camp_solver.h): pattern validation and
// preprocessing, SpMV schedules, arrangement choice and kernel launches.
#include <algorithm>
#include <cstdint>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "camp_internal.h"
#include "camp_testing.h"
#include "schedule.h"

namespace camp {
cudaError_t launch_warp_1(const WarpArgs &, int, int, size_t, cudaStream_t);
#define CAMP_DECL(E)                                                        \
  cudaError_t launch_warp_##E(const WarpArgs &, int, int, size_t, cudaStream_t); \
  cudaError_t occ_warp_##E(int, size_t, int *);
CAMP_DECL(2) CAMP_DECL(3) CAMP_DECL(4) CAMP_DECL(5) CAMP_DECL(6) CAMP_DECL(7)
CAMP_DECL(8) CAMP_DECL(9) CAMP_DECL(10) CAMP_DECL(11) CAMP_DECL(12)
CAMP_DECL(13) CAMP_DECL(14) CAMP_DECL(15) CAMP_DECL(16)
cudaError_t occ_warp_1(int, size_t, int *);
#define CAMP_DECLM(E)                                                        \
  cudaError_t launch_mixed_##E(const MixedArgs &, int, int, size_t, cudaStream_t); \
  cudaError_t occ_mixed_##E(int, size_t, int *);
CAMP_DECLM(1) CAMP_DECLM(2) CAMP_DECLM(3) CAMP_DECLM(4) CAMP_DECLM(5)
CAMP_DECLM(6) CAMP_DECLM(7) CAMP_DECLM(8) CAMP_DECLM(9) CAMP_DECLM(10)
CAMP_DECLM(11) CAMP_DECLM(12) CAMP_DECLM(13) CAMP_DECLM(14) CAMP_DECLM(15)
CAMP_DECLM(16)
#define CAMP_DECLF(E)                                                         \
  cudaError_t launch_assemble_##E(const WarpArgs &, int, int, size_t, cudaStream_t); \
  cudaError_t occ_assemble_##E(int, size_t, int *);                            \
  cudaError_t launch_newton_##E(const WarpArgs &, int, int, size_t, cudaStream_t);   \
  cudaError_t occ_newton_##E(int, size_t, int *);
CAMP_DECLF(1) CAMP_DECLF(2) CAMP_DECLF(3) CAMP_DECLF(4) CAMP_DECLF(5)
CAMP_DECLF(6) CAMP_DECLF(7) CAMP_DECLF(8)
#undef CAMP_DECLF
#undef CAMP_DECLM
#undef CAMP_DECL

cudaError_t launch_warp(int E, const WarpArgs &a, int wpb, int grid,
                        size_t smem, cudaStream_t st) {
  switch (E) {
#define C(E) case E: return launch_warp_##E(a, wpb, grid, smem, st);
    C(1) C(2) C(3) C(4) C(5) C(6) C(7) C(8) C(9) C(10) C(11) C(12) C(13)
    C(14) C(15) C(16)
#undef C
    default: return cudaErrorInvalidValue;
  }
}
static cudaError_t warp_occupancy_query(int E, int wpb, size_t smem, int *blocks) {
  switch (E) {
#define C(E) case E: return occ_warp_##E(wpb, smem, blocks);
    C(1) C(2) C(3) C(4) C(5) C(6) C(7) C(8) C(9) C(10) C(11) C(12) C(13)
    C(14) C(15) C(16)
#undef C
    default: return cudaErrorInvalidValue;
  }
}

// The occupancy of a launch shape does not change: remember the answers
// (fixed-size record, no heap allocation).
cudaError_t warp_occupancy(int E, int wpb, size_t smem, int *blocks) {
  struct Entry { int dev, E, wpb; size_t smem; int blocks; };
  static std::mutex mu;
  static Entry memo[256];
  static int nmemo = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lock(mu);
    for (int i = 0; i < nmemo; ++i)
      if (memo[i].dev == dev && memo[i].E == E && memo[i].wpb == wpb && memo[i].smem == smem) {
        *blocks = memo[i].blocks;
        return cudaSuccess;
      }
  }
  if ((e = warp_occupancy_query(E, wpb, smem, blocks)) != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (nmemo < 256) memo[nmemo++] = Entry{dev, E, wpb, smem, *blocks};
  return cudaSuccess;
}

cudaError_t launch_mixed(int E, const MixedArgs &a, int wpb, int grid,
                         size_t smem, cudaStream_t st) {
  switch (E) {
#define C(E) case E: return launch_mixed_##E(a, wpb, grid, smem, st);
    C(1) C(2) C(3) C(4) C(5) C(6) C(7) C(8) C(9) C(10) C(11) C(12) C(13)
    C(14) C(15) C(16)
#undef C
    default: return cudaErrorInvalidValue;
  }
}
cudaError_t mixed_occupancy(int E, int wpb, size_t smem, int *blocks) {
  switch (E) {
#define C(E) case E: return occ_mixed_##E(wpb, smem, blocks);
    C(1) C(2) C(3) C(4) C(5) C(6) C(7) C(8) C(9) C(10) C(11) C(12) C(13)
    C(14) C(15) C(16)
#undef C
    default: return cudaErrorInvalidValue;
  }
}

#define CAMP_DISPATCH8(fn, name)                                              \
  cudaError_t fn(int E, const WarpArgs &a, int wpb, int grid, size_t smem,      \
                 cudaStream_t st) {                                             \
    switch (E) {                                                                \
      case 1: return launch_##name##_1(a, wpb, grid, smem, st);                 \
      case 2: return launch_##name##_2(a, wpb, grid, smem, st);                 \
      case 3: return launch_##name##_3(a, wpb, grid, smem, st);                 \
      case 4: return launch_##name##_4(a, wpb, grid, smem, st);                 \
      case 5: return launch_##name##_5(a, wpb, grid, smem, st);                 \
      case 6: return launch_##name##_6(a, wpb, grid, smem, st);                 \
      case 7: return launch_##name##_7(a, wpb, grid, smem, st);                 \
      case 8: return launch_##name##_8(a, wpb, grid, smem, st);                 \
      default: return cudaErrorInvalidValue;                                    \
    }                                                                           \
  }
#define CAMP_OCCUPANCY8(fn, name)                                             \
  cudaError_t fn(int E, int wpb, size_t smem, int *blocks) {                    \
    switch (E) {                                                                \
      case 1: return occ_##name##_1(wpb, smem, blocks);                         \
      case 2: return occ_##name##_2(wpb, smem, blocks);                         \
      case 3: return occ_##name##_3(wpb, smem, blocks);                         \
      case 4: return occ_##name##_4(wpb, smem, blocks);                         \
      case 5: return occ_##name##_5(wpb, smem, blocks);                         \
      case 6: return occ_##name##_6(wpb, smem, blocks);                         \
      case 7: return occ_##name##_7(wpb, smem, blocks);                         \
      case 8: return occ_##name##_8(wpb, smem, blocks);                         \
      default: return cudaErrorInvalidValue;                                    \
    }                                                                           \
  }
CAMP_DISPATCH8(launch_assemble, assemble)
CAMP_OCCUPANCY8(assemble_occupancy, assemble)
CAMP_DISPATCH8(launch_newton, newton)
CAMP_OCCUPANCY8(newton_occupancy, newton)
#undef CAMP_DISPATCH8
#undef CAMP_OCCUPANCY8

constexpr int kHostChunks = 5;        // pipeline depth of camp_solver_solve_host
constexpr int kHostSolveStreams = 4;  // concurrent chunk solves

cudaError_t ensure_max_smem(const void *kernel) {
  // fixed-size record (no heap allocation: the allocation-free entry point
  // launches through here too)
  static std::mutex mu;
  static const void *done_kernel[512];
  static int done_dev[512];
  static int ndone = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  for (int i = 0; i < ndone; ++i)
    if (done_kernel[i] == kernel && done_dev[i] == dev) return cudaSuccess;
  int optin = 0;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin)) != cudaSuccess)
    return e;
  if (ndone < 512) {
    done_kernel[ndone] = kernel;
    done_dev[ndone] = dev;
    ++ndone;
  }
  return cudaSuccess;
}

namespace {

thread_local std::string g_err;

camp_status fail(camp_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

camp_status cuda_fail(cudaError_t e, const char *where) {
  return fail(CAMP_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

// Balanced static SpMV schedule for lanes_per_cell lanes (sched::build in
// schedule.h: whole rows bin-packed onto lanes, the entries of a row ordered
// so that a slot's gathers fall on distinct shared-memory banks).  For every
// slot: the packed word (column, row, end of row), the entry of the cell's A
// row it multiplies (src; the transposed view maps through its permutation),
// and for every row the slot of its diagonal entry.
struct Schedule {
  int Lc = 0, L = 0;
  std::vector<SchedWord> words;  // [L][Lc]
  std::vector<int> src;          // [L][Lc], -1 = padding
  std::vector<int> dslot;        // [n]
  std::vector<int> dst;          // [nnz] slot of each A entry (forward order)
  std::vector<int> padfrom;      // [Lc] first padding slot of each lane
  // automatic warps per block, found once per kernel kind (0: not yet):
  // plain solve, fused assembly, Newton corrector
  int auto_wpb[3] = {0, 0, 0};
  SchedWord *d_words = nullptr;
  int *d_src = nullptr, *d_dslot = nullptr, *d_dst = nullptr, *d_padfrom = nullptr;
  // 16 lanes per cell only: the split schedule of one cell on 32 lanes (L2
  // 0: none); see split_schedule
  int L2 = 0;
  std::vector<SchedWord> words2;  // [L2][32]
  std::vector<int> dst2, padfrom2, dslot2;
  SchedWord *d_words2 = nullptr;
  int *d_dst2 = nullptr, *d_padfrom2 = nullptr, *d_dslot2 = nullptr;
};

// The split schedule of a 16-lane schedule: one cell on all 32 lanes, lane v
// and lane v + 16 sharing the rows of 16-lane lane v, whole rows to either
// side (the subset that balances the two sides' slot counts best, found
// exhaustively for up to 16 rows, else greedily longest first); every row
// keeps its slots' order, so each row's sum is the same chain of
// multiply-adds as in the pair solve; padding slots multiply zero by column
// 0.  Fills L2, words2, dst2, padfrom2 and dslot2 (L2 stays 0 unless the
// schedule is 16 lanes wide).
void split_schedule(Schedule &S, int n, int nnz) {
  if (S.Lc != 16 || S.L == 0) return;
  std::vector<std::vector<int>> rstart(16), rlen(16);
  std::vector<std::vector<char>> side(16);  // side[v][r]: row r of lane v goes to lane v + 16
  int L2 = 1;
  for (int v = 0; v < 16; ++v) {
    const int len = S.padfrom[v];
    for (int j = 0, st = 0; j < len; ++j)
      if (S.words[(size_t)j * 16 + v] & kSlotEnd) {
        rstart[v].push_back(st);
        rlen[v].push_back(j + 1 - st);
        st = j + 1;
      }
    const int R = (int)rlen[v].size();
    side[v].assign(R, 0);
    int best = len;
    if (R <= 16) {
      unsigned bestm = 0u;
      for (unsigned msk = 0; msk < (1u << R); ++msk) {
        int l1 = 0;
        for (int r = 0; r < R; ++r)
          if ((msk >> r) & 1u) l1 += rlen[v][r];
        const int m = std::max(l1, len - l1);
        if (m < best) {
          best = m;
          bestm = msk;
        }
      }
      for (int r = 0; r < R; ++r) side[v][r] = (char)((bestm >> r) & 1u);
    } else {
      std::vector<int> ord(R);
      for (int r = 0; r < R; ++r) ord[r] = r;
      std::stable_sort(ord.begin(), ord.end(),
                       [&](int x, int y) { return rlen[v][x] > rlen[v][y]; });
      int l0 = 0, l1 = 0;
      for (int r : ord) {
        if (l1 < l0) {
          l1 += rlen[v][r];
          side[v][r] = 1;
        } else {
          l0 += rlen[v][r];
        }
      }
      best = std::max(l0, l1);
    }
    L2 = std::max(L2, best);
  }
  S.L2 = L2;
  S.words2.assign((size_t)L2 * 32, 0u);
  S.padfrom2.assign(32, 0);
  S.dst2.assign(nnz, -1);
  S.dslot2.assign(n, -1);
  std::vector<int> map16((size_t)S.L * 16, -1);
  for (int v = 0; v < 16; ++v) {
    int fill[2] = {0, 0};
    for (size_t r = 0; r < rlen[v].size(); ++r) {
      const int h = side[v][r];
      const int lane = v + 16 * h;
      for (int q = 0; q < rlen[v][r]; ++q) {
        const size_t t16 = (size_t)(rstart[v][r] + q) * 16 + v;
        const size_t t2 = (size_t)fill[h]++ * 32 + lane;
        S.words2[t2] = S.words[t16];
        map16[t16] = (int)t2;
        if (S.src[t16] >= 0) S.dst2[S.src[t16]] = (int)t2;
      }
    }
    S.padfrom2[v] = fill[0];
    S.padfrom2[v + 16] = fill[1];
  }
  for (int r = 0; r < n; ++r)
    if (S.dslot[r] >= 0) S.dslot2[r] = map16[S.dslot[r]];
}

Schedule build_schedule(int n, const std::vector<int> &rp,
                        const std::vector<int> &ci, const std::vector<int> &perm,
                        const std::vector<int> &diag, int Lc) {
  std::vector<int> order(n), bin_rows((size_t)Lc * n), bin_count(Lc), cursor(Lc), cur_row(Lc),
      rem((size_t)Lc * n), rem_count(Lc);
  std::vector<long> load(Lc);
  const sched::Work w = {order.data(), load.data(), bin_rows.data(), bin_count.data(),
                         cursor.data(), cur_row.data(), rem.data(), rem_count.data()};
  long total = 0;  // an upper bound of L * Lc: every row on one lane
  for (int r = 0; r < n; ++r) total += rp[r + 1] - rp[r];
  std::vector<SchedWord> words((size_t)total * Lc);
  std::vector<int> entry((size_t)total * Lc);
  Schedule S;
  S.Lc = Lc;
  S.dslot.assign(n, -1);
  S.padfrom.assign(Lc, 0);
  S.L = sched::build(n, rp.data(), ci.data(), diag.data(), Lc, words.size(), w, words.data(),
                     entry.data(), S.dslot.data(), S.padfrom.data());
  const size_t slots = (size_t)S.L * Lc;
  S.words.assign(words.begin(), words.begin() + slots);
  S.src.assign(slots, -1);
  S.dst.assign(rp[n], -1);
  for (size_t t = 0; t < slots; ++t) {
    if (entry[t] < 0) continue;
    S.src[t] = perm.empty() ? entry[t] : perm[entry[t]];
    S.dst[S.src[t]] = (int)t;
  }
  return S;
}

// one orientation of the pattern: forward (A) or transposed (A^T)
struct View {
  int n = 0, nnz = 0;
  std::vector<int> rp, ci, diag, perm;  // perm empty for the forward view
  int *d_rp = nullptr, *d_ci = nullptr, *d_diag = nullptr, *d_perm = nullptr;
  std::map<int, Schedule> sched;  // by lanes per cell
};

template <class T>
cudaError_t upload(T **dst, const std::vector<T> &src) {
  *dst = nullptr;
  if (src.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc((void **)dst, src.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src.data(), src.size() * sizeof(T),
                    cudaMemcpyHostToDevice);
}

// Mass-action mechanism attached to a handle for the fused assembly: its
// Jacobian terms in reaction order (pattern entry, concentration factor,
// signed rate constant) and, per lanes-per-cell choice, the terms grouped by
// schedule slot on the device.
struct MechTerms {
  int count = 0;               // Jacobian terms per lane (padded)
  int *d_tmeta = nullptr;
  double *d_tval = nullptr;
  int rcount = 0;              // rate terms per lane (padded)
  int *d_rmeta = nullptr;
  double *d_rval = nullptr;
  void release() {
    cudaFree(d_tmeta);
    cudaFree(d_tval);
    cudaFree(d_rmeta);
    cudaFree(d_rval);
  }
};
struct Mechanism {
  int R = 0;
  std::vector<int> entry, spec;  // Jacobian terms: CSR entry, factor species
  std::vector<double> val;
  std::vector<int> rrow, ra, rb;  // rate terms: row of f, factor species
  std::vector<double> rk;         // signed rate constant
  std::map<int, MechTerms> by_lanes;
};

}  // namespace
}  // namespace camp

using namespace camp;

struct camp_solver {
  int device = 0, sms = 0;
  size_t smem_optin = 0;
  int n = 0, nnz = 0;
  cudaStream_t stream = nullptr;
  View fwd, tr;
  int *d_row_of = nullptr;  // forward view: row of entry k
  // dynamic group queues of the warp kernel, one pair per stream the handle
  // uses: pair 0 its own stream, pairs 1.. the solve streams of solve_host
  unsigned int *d_queue = nullptr;
  int arrangement = CAMP_ARR_AUTO, lanes = 0, cpb = 1, wpb = 0;
  // staging for camp_solver_solve_host
  double *h_dA = nullptr, *h_db = nullptr, *h_dx = nullptr, *h_dres = nullptr;
  int *h_dit = nullptr, *h_dst = nullptr;
  size_t h_cap_cells = 0;
  // solve_host pipeline: [0] host-to-device copies, [1] device-to-host
  // copies, [2 ..] solves (round robin, so the solves of consecutive chunks
  // overlap); per chunk an event after its input copy and one after its solve
  cudaStream_t h_streams[2 + kHostSolveStreams] = {};
  cudaEvent_t h_in[kHostChunks] = {}, h_done[kHostChunks] = {}, h_start = nullptr;
  std::mutex mu;
  Mechanism mech;
  // difficulty ordering (camp_solver_set_ordering): scratch grown on demand;
  // the in-launch ordering's workspace follows the queue pairs in d_queue,
  // its time-out word is host-mapped (allocated on first use)
  int ordering = 1;
  void *d_order_scratch = nullptr;
  size_t order_cap = 0;  // bytes
  int *h_ord_err = nullptr, *d_ord_err = nullptr;
  // rows the in-launch ordering samples: picked on the host from the peak
  // rows a full-diagonal ("calibration") launch records, read back without
  // blocking (pinned copy + event); nsamp 0: no sample yet
  unsigned *d_hits = nullptr, *h_hits = nullptr;
  // in-launch order ([cells] entries, all zero between launches) and the
  // class words of CTAs whose share exceeds one pass ([cells])
  int *d_ord = nullptr;
  size_t ord_cap = 0;  // cells
  int *d_samp = nullptr;
  int nsamp = 0;
  cudaEvent_t ev_hits = nullptr;
  bool hits_pending = false;
  unsigned ordered_solves = 0;
  // limit of the in-launch ordering's waits (SM cycles) and, for tests, a
  // switch that treats every cooperative launch as refused
  long long ord_wait = kOrdWaitCycles;
  int refuse_cooperative = 0;
  // single-cell tickets of the plain 16-lane launch: < 0 automatic, else the
  // number of tail pairs solved as single cells (camp_solver_set_single_tail)
  int single_tail = -1;
};

namespace {

cudaError_t view_schedule(View &v, int Lc, Schedule **out) {
  auto it = v.sched.find(Lc);
  if (it == v.sched.end()) {
    Schedule S = build_schedule(v.n, v.rp, v.ci, v.perm, v.diag, Lc);
    split_schedule(S, v.n, v.nnz);
    cudaError_t e = upload(&S.d_words, S.words);
    if (e == cudaSuccess) e = upload(&S.d_src, S.src);
    if (e == cudaSuccess) e = upload(&S.d_dslot, S.dslot);
    if (e == cudaSuccess) e = upload(&S.d_dst, S.dst);
    if (e == cudaSuccess) e = upload(&S.d_padfrom, S.padfrom);
    if (e == cudaSuccess && S.L2) e = upload(&S.d_words2, S.words2);
    if (e == cudaSuccess && S.L2) e = upload(&S.d_dst2, S.dst2);
    if (e == cudaSuccess && S.L2) e = upload(&S.d_padfrom2, S.padfrom2);
    if (e == cudaSuccess && S.L2) e = upload(&S.d_dslot2, S.dslot2);
    if (e != cudaSuccess) {
      cudaFree(S.d_words);
      cudaFree(S.d_src);
      cudaFree(S.d_dslot);
      cudaFree(S.d_dst);
      cudaFree(S.d_padfrom);
      cudaFree(S.d_words2);
      cudaFree(S.d_dst2);
      cudaFree(S.d_padfrom2);
      cudaFree(S.d_dslot2);
      return e;
    }
    it = v.sched.emplace(Lc, std::move(S)).first;
  }
  *out = &it->second;
  return cudaSuccess;
}

void free_view(View &v) {
  cudaFree(v.d_rp);
  cudaFree(v.d_ci);
  cudaFree(v.d_diag);
  cudaFree(v.d_perm);
  for (auto &kv : v.sched) {
    cudaFree(kv.second.d_words);
    cudaFree(kv.second.d_src);
    cudaFree(kv.second.d_dslot);
    cudaFree(kv.second.d_dst);
    cudaFree(kv.second.d_padfrom);
    cudaFree(kv.second.d_words2);
    cudaFree(kv.second.d_dst2);
    cudaFree(kv.second.d_padfrom2);
    cudaFree(kv.second.d_dslot2);
  }
  v.sched.clear();
}

int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

// Doubles from one cell's shared-memory block to the next: at least `need`,
// and Lc = 32/k doubles modulo 16 (one pass over the 32 four-byte banks), so
// that the 16/Lc cells that share a half-warp, which read the same relative
// addresses in the same instruction, sit Lc bank pairs apart: their
// consecutive accesses (Lc doubles per cell) tile the 16 bank pairs, and the
// schedule's gathers (columns of distinct residues modulo Lc, schedule.h)
// stay conflict-free.
int bank_spread_stride(int need, int k) {
  const int want = (32 / k) % 16;
  int s = need;
  while (s % 16 != want) ++s;
  return s;
}

// Warp kernel shared-memory bytes for one CTA.
size_t warp_smem(const View &v, int Lc, int L, int wpb, int *segA, int *segV,
                 int *segStride, int extra_vectors = 0) {
  const int k = 32 / Lc;
  const int E = (v.n + Lc - 1) / Lc;
  *segA = (L * Lc + 1) & ~1;  // A in slot order
  *segV = ((E * Lc + 1) + 1) & ~1;
  *segStride = bank_spread_stride(*segA + (warp_vectors(E) + extra_vectors) * *segV, k);
  const size_t sch = sched_smem_bytes(L * Lc);
  return sch + (size_t)wpb * k * (size_t)*segStride * 8;
}

// Warps per block of an automatic warp-packed launch: the most resident
// warps per SM (the CTA's schedule copy and its warps' cell regions must pack
// into the SM's shared memory; occ gives the CTAs per SM of the kernel), 4
// unless another count fits more.  Fills the shared-memory layout.
typedef cudaError_t (*OccFn)(int E, int wpb, size_t smem, int *blocks);
cudaError_t pick_warps_per_block(const View &v, int Lc, int L, int E, int extra_vectors,
                                 size_t optin, OccFn occ_fn, int *cache, int *wpb, size_t *smem,
                                 int *segA, int *segV, int *segStride) {
  if (*cache > 0) {
    *wpb = *cache;
    *smem = warp_smem(v, Lc, L, *wpb, segA, segV, segStride, extra_vectors);
    return cudaSuccess;
  }
  int best = -1;
  for (int w : {4, 8, 6, 5, 3, 2, 1}) {
    int sa = 0, sv = 0, ss = 0, occ = 0;
    const size_t sm = warp_smem(v, Lc, L, w, &sa, &sv, &ss, extra_vectors);
    if (sm > optin) continue;
    const cudaError_t e = occ_fn(E, w, sm, &occ);
    if (e != cudaSuccess) return e;
    if (occ * w > best) {
      best = occ * w;
      *wpb = w;
    }
  }
  if (best < 0) {
    *smem = optin + 1;  // does not fit even with one warp
    return cudaSuccess;
  }
  *cache = *wpb;
  *smem = warp_smem(v, Lc, L, *wpb, segA, segV, segStride, extra_vectors);
  return cudaSuccess;
}

size_t mixed_smem(const View &v, int Lc, int L, int wpb, int *segA, int *segV, bool a64_smem) {
  const int k = 32 / Lc;
  const int E = (v.n + Lc - 1) / Lc;
  *segA = (L * Lc + 1) & ~1;  // A in slot order
  *segV = ((E * Lc + 1) + 1) & ~1;
  const size_t sch = sched_smem_bytes(L * Lc);
  return sch + (size_t)wpb * k * ((size_t)(a64_smem ? 12 : 4) * *segA + (size_t)28 * *segV);
}

// Automatic arrangement: the most cells per warp (fewest lanes per cell) that
// keeps at most `rows` rows per lane; FP64 scalar work and reductions are
// shared by the cells of a warp, while per-lane rows cost registers.
constexpr int kAutoRowsPerLane = 5;
constexpr int kAutoRowsPerLaneMixed = 3;
int auto_lanes(int n, int rows) {
  for (int cand = 1; cand <= 32; cand *= 2)
    if ((n + cand - 1) / cand <= rows) return cand;
  return (n + 31) / 32 <= kMaxE ? 32 : 0;
}

size_t block_smem(int n, int nnz, int cpb, int threads) {
  return ((size_t)cpb * nnz + 3 * (size_t)cpb * n + 3 * (size_t)threads +
          3 * (size_t)cpb) * 8;
}

// Stride of the first wave's ticket-to-group map: coprime with the wave (a
// bijection) and near the golden section of it, so that any run of
// consecutive tickets lands on groups spread over the whole difficulty range.
int spread_stride(int wave) {
  if (wave <= 2) return 1;
  const int s0 = (int)(0.6180339887 * wave);
  for (int d = 0; d < wave; ++d) {
    for (int s : {s0 - d, s0 + d})
      if (s >= 1 && s < wave && std::gcd(s, wave) == 1) return s;
  }
  return 1;
}

// Device and host state of the in-launch ordering, allocated on first use:
// the host-mapped time-out word, the peak-row counts (device and pinned
// host copies), the sampled positions and the read-back event.
cudaError_t ordering_state(camp_solver_t h) {
  // each piece allocated once: a call after a failed one completes the rest
  cudaError_t e = cudaSuccess;
  if (!h->h_ord_err) {
    if ((e = cudaHostAlloc(&h->h_ord_err, sizeof(int), cudaHostAllocMapped)) != cudaSuccess)
      return e;
    *h->h_ord_err = 0;
  }
  if (!h->d_ord_err &&
      (e = cudaHostGetDevicePointer(&h->d_ord_err, h->h_ord_err, 0)) != cudaSuccess)
    return e;
  if (h->n <= kOrdSample) return cudaSuccess;  // the whole diagonal is the sample
  if (!h->d_hits && (e = cudaMalloc(&h->d_hits, (size_t)h->n * sizeof(unsigned))) != cudaSuccess)
    return e;
  if (!h->d_samp && (e = cudaMalloc(&h->d_samp, kOrdSample * sizeof(int))) != cudaSuccess)
    return e;
  if (!h->h_hits && (e = cudaHostAlloc(&h->h_hits, (size_t)h->n * sizeof(unsigned),
                                       cudaHostAllocDefault)) != cudaSuccess)
    return e;
  if (!h->ev_hits &&
      (e = cudaEventCreateWithFlags(&h->ev_hits, cudaEventDisableTiming)) != cudaSuccess)
    return e;
  return cudaSuccess;
}

// Once a calibration launch's peak-row counts have reached the host, sample
// the (up to kOrdSample) rows where the most CTAs' hardest cells peaked.
cudaError_t pick_sample(camp_solver_t h, cudaStream_t st) {
  if (!h->hits_pending) return cudaSuccess;
  cudaError_t e = cudaEventQuery(h->ev_hits);
  if (e == cudaErrorNotReady) return cudaSuccess;
  if (e != cudaSuccess) return e;
  h->hits_pending = false;
  std::vector<int> rows;
  for (int i = 0; i < h->n; ++i)
    if (h->h_hits[i]) rows.push_back(i);
  std::stable_sort(rows.begin(), rows.end(),
                   [&](int p, int q) { return h->h_hits[p] > h->h_hits[q]; });
  if (rows.size() > (size_t)kOrdSample) rows.resize(kOrdSample);
  if (rows.empty()) return cudaSuccess;
  int pos[kOrdSample];
  for (size_t j = 0; j < rows.size(); ++j) pos[j] = h->fwd.diag[rows[j]];
  // a pageable source: the copy is staged before the call returns
  e = cudaMemcpyAsync(h->d_samp, pos, rows.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  h->nsamp = (int)rows.size();
  return cudaSuccess;
}

// The separate ordering pass (a memset, a classify and a scatter launch):
// a.order points at its result.
template <class Args>
camp_status separate_ordering(camp_solver_t h, Args &a, const double *A_vals, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  const size_t need = difficulty_scratch_bytes(a.cells);
  if (need > h->order_cap) {
    cudaFree(h->d_order_scratch);
    h->d_order_scratch = nullptr;
    h->order_cap = 0;
    if ((e = cudaMalloc(&h->d_order_scratch, need)) != cudaSuccess)
      return fail(CAMP_ENOMEM, "ordering scratch: %s", cudaGetErrorString(e));
    h->order_cap = need;
  }
  int *order = nullptr;
  e = launch_difficulty_order(A_vals, a.cells, h->fwd.n, h->fwd.nnz, h->fwd.d_diag,
                              h->d_order_scratch, &order, st);
  if (e != cudaSuccess) return cuda_fail(e, "difficulty ordering");
  a.order = order;
  return CAMP_OK;
}

// A cooperative launch was refused as too large (the GPU offers fewer SMs
// than the occupancy query assumed, e.g. a partitioned GPU): order by the
// separate pass instead and clear the in-launch fields.  The refused launch
// ran nothing, so the order entries and the workspace are still zero.
template <class Args>
camp_status fall_back_to_separate_ordering(camp_solver_t h, Args &a, const double *A_vals,
                                           cudaStream_t st) {
  (void)cudaGetLastError();
  a.ord_out = nullptr;
  a.ord_ws = nullptr;
  a.ord_cls = nullptr;
  a.ord_rows = nullptr;
  a.ord_nrows = 0;
  a.ord_hits = nullptr;
  a.ord_err = nullptr;
  return separate_ordering(h, a, A_vals, st);
}

// The in-launch order's entries and class words for `cells` cells ([cells]
// each), grown on demand; the entries start (and every launch leaves them)
// all zero.
camp_status ensure_order_capacity(camp_solver_t h, int cells, cudaStream_t st) {
  if ((size_t)cells <= h->ord_cap) return CAMP_OK;
  cudaFree(h->d_ord);
  h->d_ord = nullptr;
  h->ord_cap = 0;
  cudaError_t e;
  if ((e = cudaMalloc(&h->d_ord, (size_t)cells * 2 * sizeof(int))) != cudaSuccess)
    return fail(CAMP_ENOMEM, "ordering scratch: %s", cudaGetErrorString(e));
  if ((e = cudaMemsetAsync(h->d_ord, 0, (size_t)cells * sizeof(int), st)) != cudaSuccess)
    return cuda_fail(e, "ordering scratch");
  h->ord_cap = (size_t)cells;
  return CAMP_OK;
}

// In-launch ordering of the fused-assembly and Newton launches (orderings 1
// and 2): cells classified by gamma, as the plain launch classifies them by
// its sampled diagonal (there is no matrix before a cell is assembled).
// Leaves a unordered when the warp regions cannot lend the ordering its
// shared memory.
camp_status setup_gamma_ordering(camp_solver_t h, WarpArgs &a, size_t smem_free,
                                 cudaStream_t st) {
  if (!h->ordering || a.cells <= 1 || smem_free < kOrdSmemBytes) return CAMP_OK;
  camp_status rs = ensure_order_capacity(h, a.cells, st);
  if (rs != CAMP_OK) return rs;
  cudaError_t e;
  if ((e = ordering_state(h)) != cudaSuccess) return cuda_fail(e, "ordering state");
  a.ord_out = h->d_ord;
  a.ord_cls = h->d_ord + h->ord_cap;
  a.ord_ws = (int *)(h->d_queue + 2 * (1 + kHostSolveStreams));
  a.ord_err = h->d_ord_err;
  a.ord_wait = h->ord_wait;
  a.order = a.ord_out;
  a.ord_rows = nullptr;
  a.ord_nrows = 1;
  a.ord_hits = nullptr;
  return CAMP_OK;
}

// A refused cooperative launch of an ordered fused launch runs in index order.
void drop_gamma_ordering(WarpArgs &a) {
  (void)cudaGetLastError();
  a.ord_out = nullptr;
  a.ord_ws = nullptr;
  a.ord_cls = nullptr;
  a.ord_err = nullptr;
  a.order = nullptr;
  a.ord_wave = a.ord_stride = 0;
}

// Difficulty ordering of a warp-packed solve on the handle's own stream (one
// workspace per handle).  Ordering 1 runs inside the (cooperative) solve
// launch, borrowing kOrdSmemBytes of the warp regions (smem_free bytes of
// them) before they are used; ordering 2, or 1 where that does not fit, runs
// the separate classify and scatter pass.  Fills the order fields of a
// (WarpArgs or MixedArgs; a.cells, a.ngroups set); *calibrate tells the
// caller to read the peak-row counts back after the launch.
template <class Args>
camp_status setup_ordering(camp_solver_t h, Args &a, const double *A_vals, size_t smem_free,
                           cudaStream_t st, bool *calibrate) {
  const int cells = a.cells;
  *calibrate = false;
  if (!h->ordering || cells <= 1) return CAMP_OK;
  cudaError_t e = cudaSuccess;
  const bool inl = h->ordering == 1 && smem_free >= kOrdSmemBytes;
  if (inl) {
    const camp_status rs = ensure_order_capacity(h, cells, st);
    if (rs != CAMP_OK) return rs;
  }
  if (!inl) return separate_ordering(h, a, A_vals, st);
  if ((e = ordering_state(h)) != cudaSuccess) return cuda_fail(e, "ordering state");
  a.ord_out = h->d_ord;
  a.ord_cls = h->d_ord + h->ord_cap;
  a.ord_ws = (int *)(h->d_queue + 2 * (1 + kHostSolveStreams));
  a.ord_err = h->d_ord_err;
  a.ord_wait = h->ord_wait;
  a.order = a.ord_out;
  // the diagonal is the same in both orientations: forward positions
  a.ord_rows = h->fwd.d_diag;
  a.ord_nrows = h->n;
  if (h->n <= kOrdSample) return CAMP_OK;
  // under stream capture the sample stays as it is (no host read-back)
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if ((e = cudaStreamIsCapturing(st, &cap)) != cudaSuccess) return cuda_fail(e, "capture query");
  if (cap == cudaStreamCaptureStatusNone) {
    if ((e = pick_sample(h, st)) != cudaSuccess) return cuda_fail(e, "ordering sample");
    if (!h->hits_pending && (h->nsamp == 0 || h->ordered_solves % kOrdRecalibrate == 0)) {
      *calibrate = true;
      if ((e = cudaMemsetAsync(h->d_hits, 0, (size_t)h->n * sizeof(unsigned), st)) != cudaSuccess)
        return cuda_fail(e, "ordering hits");
      a.ord_hits = h->d_hits;
    }
    ++h->ordered_solves;
  }
  if (!*calibrate && h->nsamp > 0) {
    a.ord_rows = h->d_samp;
    a.ord_nrows = h->nsamp;
  }
  return CAMP_OK;
}

// After a calibrating launch: the peak-row counts come back without
// blocking; a later solve picks the rows up.
camp_status read_back_hits(camp_solver_t h, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(h->h_hits, h->d_hits, (size_t)h->n * sizeof(unsigned),
                                  cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_hits, st);
  if (e != cudaSuccess) return cuda_fail(e, "ordering hits read-back");
  h->hits_pending = true;
  return CAMP_OK;
}

// The first wave of an ordered launch (WarpArgs::ord_wave): stratified when
// every warp of the grid gets a group, else tickets spread over the order.
template <class Args>
void set_wave(Args &a, int grid, int wpb) {
  if (!a.order) return;
  if (a.ngroups >= grid * wpb) {
    a.ord_wave = grid * wpb;
    a.ord_stride = 0;
  } else {
    a.ord_wave = a.ngroups;
    a.ord_stride = spread_stride(a.ngroups);
  }
}

// The cooperative launch of an ordered solve (or its refusal, which a test
// can force so that the fallback below runs on any GPU).
template <class Launch>
cudaError_t launch_cooperative(camp_solver_t h, bool cooperative, Launch launch) {
  if (cooperative && h->refuse_cooperative) return cudaErrorCooperativeLaunchTooLarge;
  return launch();
}

// Single-cell tickets of a plain launch at 16 lanes per cell (warp_single.cuh):
// the last R pairs of the launch become 2R single-cell tickets.  Automatic R
// (measured at 80 species on 152 SMs x 16 warps): every pair when the pairs
// would keep at most a quarter of the resident warps busy (a lone warp's
// latency decides such a launch: 60 against 75 us at 64 to 608 cells, 65.5
// against 75.8 at 1,212), else none (at full load one cell per warp costs
// about 13 % more per cell, and turning the pairs past the last full wave
// into singles measured within the noise at 10,000 cells).
// camp_solver_set_single_tail overrides it.  Sets
// single_from, ngroups (tickets) and the split schedule's arguments; leaves
// the launch without single tickets when the split schedule does not fit
// the warp's region.
void set_single_tickets(camp_solver_t h, const Schedule &S, WarpArgs &a, int wpb, int occ) {
  const int pairs = a.ngroups;
  a.single_from = pairs;
  a.sched2 = nullptr;
  if (S.L2 == 0 || a.Lc != 16 || a.k != 2 || h->single_tail == 0) return;
  const int E16 = (a.n + 15) / 16;
  const size_t need = ((size_t)(S.L2 * 32 + 1) & ~(size_t)1) + 3 * (size_t)(((16 * E16 + 1) + 1) & ~1);
  if (E16 > kRegVecMaxE || need > 2 * (size_t)a.segStride) return;
  const long resident = (long)h->sms * occ * wpb;  // warps the GPU holds at once
  int R = 0;
  if (h->single_tail > 0) {
    R = std::min(pairs, h->single_tail);
  } else if (4L * pairs <= resident) {
    R = pairs;  // a small batch: every cell alone, each warp nearly so
  }
  if (R == 0) return;
  const int P = pairs - R;
  a.single_from = P;
  a.ngroups = P + std::max(0, a.cells - 2 * P);
  a.L2 = S.L2;
  a.sched2 = S.d_words2;
  a.dst2 = S.d_dst2;
  a.padfrom2 = S.d_padfrom2;
  a.dslot2 = S.d_dslot2;
}

camp_status do_solve(camp_solver_t h, int cells, const double *A_vals,
                     const double *b, double *x, double tol, int maxit,
                     int *iters_out, double *resid_out, int *status_out,
                     int flags, cudaStream_t st, int queue_slot) {
  if (!h) return fail(CAMP_EINVAL, "null solver handle");
  if (cells < 0) return fail(CAMP_EINVAL, "cells < 0");
  if (!(tol > 0.0) || !std::isfinite(tol)) return fail(CAMP_EINVAL, "tol must be finite and > 0");
  if (maxit < 1) return fail(CAMP_EINVAL, "maxit must be >= 1");
  if (flags & ~(CAMP_TRANSPOSE | CAMP_X0_GIVEN)) return fail(CAMP_EINVAL, "unknown flags 0x%x", flags);
  if (cells == 0) return CAMP_OK;
  if (!A_vals || !b || !x || !iters_out || !resid_out)
    return fail(CAMP_EINVAL, "null array pointer");
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  View &v = (flags & CAMP_TRANSPOSE) ? h->tr : h->fwd;

  int arr = h->arrangement;
  int Lc = h->lanes;
  if (arr == CAMP_ARR_AUTO) {
    arr = CAMP_ARR_WARP;
    Lc = auto_lanes(v.n, kAutoRowsPerLane);
    if (Lc == 0) arr = CAMP_ARR_BLOCK;
  }

  if (arr == CAMP_ARR_WARP) {
    const int E = (v.n + Lc - 1) / Lc;
    if (E > kMaxE)
      return fail(CAMP_EUNSUPPORTED, "n=%d needs %d rows per lane at %d lanes per cell (max %d)",
                  v.n, E, Lc, kMaxE);
    Schedule *S = nullptr;
    e = view_schedule(v, Lc, &S);
    if (e != cudaSuccess) return cuda_fail(e, "schedule upload");
    int wpb = h->wpb > 0 ? h->wpb : 4;
    int segA = 0, segV = 0, segStride = 0;
    size_t smem = warp_smem(v, Lc, S->L, wpb, &segA, &segV, &segStride);
    while (smem > h->smem_optin && wpb > 1) {
      --wpb;
      smem = warp_smem(v, Lc, S->L, wpb, &segA, &segV, &segStride);
    }
    if (smem > h->smem_optin)
      return fail(CAMP_EUNSUPPORTED, "cell does not fit in shared memory (%zu bytes)", smem);
    if (h->wpb == 0 &&
        (e = pick_warps_per_block(v, Lc, S->L, E, 0, h->smem_optin, warp_occupancy,
                                  &S->auto_wpb[0], &wpb, &smem, &segA, &segV, &segStride)) !=
            cudaSuccess)
      return cuda_fail(e, "occupancy");
    WarpArgs a = {};
    a.cells = cells; a.n = v.n; a.nnz = v.nnz;
    a.Lc = Lc; a.log2Lc = ilog2(Lc); a.k = 32 / Lc; a.L = S->L;
    a.segA = segA; a.segV = segV; a.segStride = segStride;
    a.ngroups = (cells + a.k - 1) / a.k;
    a.A = A_vals; a.b = b; a.x = x; a.iters = iters_out; a.resid = resid_out;
    a.status = status_out; a.sched = S->d_words; a.src = S->d_src;
    a.dst = S->d_dst; a.padfrom = S->d_padfrom;
    a.dslot = S->d_dslot; a.tol = tol; a.maxit = maxit;
    a.x0_given = (flags & CAMP_X0_GIVEN) ? 1 : 0;
    a.queue = h->d_queue + 2 * queue_slot;
    a.order = nullptr;
    bool calibrate = false;
    int occ = 0;
    e = warp_occupancy(E, wpb, smem, &occ);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy");
    if (occ < 1) occ = 1;
    set_single_tickets(h, *S, a, wpb, occ);
    if (queue_slot == 0) {
      const camp_status rs = setup_ordering(h, a, A_vals, smem - sched_smem_bytes(S->L * Lc), st,
                                            &calibrate);
      if (rs != CAMP_OK) return rs;
    }
    const int need = (a.ngroups + wpb - 1) / wpb;
    const int grid = std::max(1, std::min(need, h->sms * occ));
    set_wave(a, grid, wpb);
    e = launch_cooperative(h, a.ord_ws != nullptr,
                           [&] { return launch_warp(E, a, wpb, grid, smem, st); });
    if (e == cudaErrorCooperativeLaunchTooLarge && a.ord_ws) {
      const camp_status rs = fall_back_to_separate_ordering(h, a, A_vals, st);
      if (rs != CAMP_OK) return rs;
      calibrate = false;
      e = launch_warp(E, a, wpb, grid, smem, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "warp kernel launch");
    return calibrate ? read_back_hits(h, st) : CAMP_OK;
  }

  // block arrangement
  const int cpb = std::max(1, h->cpb);
  const int threads = ((cpb * v.n + 31) / 32) * 32;
  if (threads > 1024)
    return fail(CAMP_EUNSUPPORTED, "cells_per_block*n = %d exceeds 1024 threads", cpb * v.n);
  const size_t smem = block_smem(v.n, v.nnz, cpb, threads);
  if (smem > h->smem_optin)
    return fail(CAMP_EUNSUPPORTED, "block does not fit in shared memory (%zu bytes)", smem);
  BlockArgs a = {};
  a.cells = cells; a.n = v.n; a.nnz = v.nnz; a.cpb = cpb;
  a.A = A_vals; a.b = b; a.x = x; a.iters = iters_out; a.resid = resid_out;
  a.status = status_out; a.a_perm = v.d_perm; a.diag = v.d_diag;
  a.row_ptr = v.d_rp; a.col_idx = v.d_ci; a.tol = tol; a.maxit = maxit;
  a.x0_given = (flags & CAMP_X0_GIVEN) ? 1 : 0;
  a.coupled = (arr == CAMP_ARR_BLOCK_COUPLED) ? 1 : 0;
  e = launch_block(a, threads, smem, st);
  if (e != cudaSuccess) return cuda_fail(e, "block kernel launch");
  return CAMP_OK;
}

}  // namespace

extern "C" {

const char *camp_last_error(void) { return g_err.c_str(); }
const char *camp_version(void) { return "campsolve 0.17 (sm_103a)"; }

camp_status camp_schedule_build(int n, int nnz, const int *row_ptr,
                                const int *col_idx, int lanes_per_cell,
                                unsigned *words, int capacity_slots,
                                int *slots_per_lane) {
  if (!row_ptr || !col_idx || !slots_per_lane)
    return fail(CAMP_EINVAL, "null argument");
  if (n < 1 || n > 1024 || nnz < n || nnz > 65535 || row_ptr[n] != nnz)
    return fail(CAMP_EINVAL, "bad sizes");
  if (lanes_per_cell < 1 || lanes_per_cell > 32 ||
      (lanes_per_cell & (lanes_per_cell - 1)))
    return fail(CAMP_EINVAL, "lanes_per_cell must be a power of two in [1, 32]");
  if (row_ptr[0] != 0) return fail(CAMP_EPATTERN, "row_ptr[0] must be 0");
  for (int i = 0; i < n; ++i)
    if (row_ptr[i + 1] < row_ptr[i] || row_ptr[i + 1] > nnz)
      return fail(CAMP_EPATTERN, "row_ptr not nondecreasing within [0, nnz] at row %d", i);
  std::vector<int> rp(row_ptr, row_ptr + n + 1), ci(col_idx, col_idx + nnz), diag(n, -1);
  for (int i = 0; i < n; ++i) {
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      if (ci[k] < 0 || ci[k] >= n)
        return fail(CAMP_EPATTERN, "column %d out of range at entry %d", ci[k], k);
      if (ci[k] == i) diag[i] = k;
    }
    if (diag[i] < 0) return fail(CAMP_EPATTERN, "diagonal entry missing in row %d", i);
  }
  Schedule S = build_schedule(n, rp, ci, std::vector<int>(), diag, lanes_per_cell);
  *slots_per_lane = S.L;
  if (words) {
    if ((long)S.L * lanes_per_cell > (long)capacity_slots)
      return fail(CAMP_EINVAL, "capacity %d < %d slots", capacity_slots,
                  S.L * lanes_per_cell);
    for (size_t q = 0; q < S.words.size(); ++q) {
      words[2 * q] = (unsigned)S.src[q];
      words[2 * q + 1] = S.words[q];
    }
  }
  return CAMP_OK;
}

camp_status camp_schedule_build_split(int n, int nnz, const int *row_ptr,
                                      const int *col_idx, unsigned *words,
                                      int capacity_slots, int *slots_per_lane) {
  if (!row_ptr || !col_idx || !slots_per_lane) return fail(CAMP_EINVAL, "null argument");
  if (n < 1 || n > 1024 || nnz < n || nnz > 65535 || row_ptr[n] != nnz)
    return fail(CAMP_EINVAL, "bad sizes");
  if ((n + 15) / 16 > 5) return fail(CAMP_EUNSUPPORTED, "more than 5 rows per lane at 16 lanes");
  if (row_ptr[0] != 0) return fail(CAMP_EPATTERN, "row_ptr[0] must be 0");
  for (int i = 0; i < n; ++i)
    if (row_ptr[i + 1] < row_ptr[i] || row_ptr[i + 1] > nnz)
      return fail(CAMP_EPATTERN, "row_ptr not nondecreasing within [0, nnz] at row %d", i);
  std::vector<int> rp(row_ptr, row_ptr + n + 1), ci(col_idx, col_idx + nnz), diag(n, -1);
  for (int i = 0; i < n; ++i) {
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      if (ci[k] < 0 || ci[k] >= n)
        return fail(CAMP_EPATTERN, "column %d out of range at entry %d", ci[k], k);
      if (ci[k] == i) diag[i] = k;
    }
    if (diag[i] < 0) return fail(CAMP_EPATTERN, "diagonal entry missing in row %d", i);
  }
  Schedule S = build_schedule(n, rp, ci, std::vector<int>(), diag, 16);
  split_schedule(S, n, nnz);
  *slots_per_lane = S.L2;
  if (words) {
    if ((long)S.L2 * 32 > (long)capacity_slots)
      return fail(CAMP_EINVAL, "capacity %d < %d slots", capacity_slots, S.L2 * 32);
    std::vector<unsigned> entry((size_t)S.L2 * 32, 0xFFFFFFFFu);
    for (int k = 0; k < nnz; ++k)
      if (S.dst2[k] >= 0) entry[S.dst2[k]] = (unsigned)k;
    for (size_t q = 0; q < S.words2.size(); ++q) {
      words[2 * q] = entry[q];
      words[2 * q + 1] = S.words2[q];
    }
  }
  return CAMP_OK;
}

camp_status camp_solver_create(camp_solver_t *out, int n, int nnz,
                               const int *row_ptr, const int *col_idx) {
  if (!out) return fail(CAMP_EINVAL, "null output handle pointer");
  *out = nullptr;
  if (!row_ptr || !col_idx) return fail(CAMP_EINVAL, "null pattern array");
  if (n < 1 || n > 1024) return fail(CAMP_EINVAL, "n=%d outside [1, 1024]", n);
  if (nnz < n || nnz > 65535) return fail(CAMP_EINVAL, "nnz=%d outside [n, 65535]", nnz);
  if (row_ptr[0] != 0 || row_ptr[n] != nnz)
    return fail(CAMP_EPATTERN, "row_ptr[0] must be 0 and row_ptr[n] must equal nnz");
  std::vector<int> diag(n, -1);
  for (int i = 0; i < n; ++i) {
    if (row_ptr[i + 1] < row_ptr[i]) return fail(CAMP_EPATTERN, "row_ptr decreases at row %d", i);
    if (row_ptr[i + 1] > nnz) return fail(CAMP_EPATTERN, "row_ptr[%d] exceeds nnz", i + 1);
    for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      const int j = col_idx[k];
      if (j < 0 || j >= n) return fail(CAMP_EPATTERN, "column %d out of range at entry %d", j, k);
      if (k > row_ptr[i] && j <= col_idx[k - 1])
        return fail(CAMP_EPATTERN, "columns not strictly increasing in row %d", i);
      if (j == i) diag[i] = k;
    }
    if (diag[i] < 0) return fail(CAMP_EPATTERN, "diagonal entry missing in row %d", i);
  }
  camp_solver *h = new (std::nothrow) camp_solver();
  if (!h) return fail(CAMP_ENOMEM, "host allocation failed");
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaGetDevice"); }
  int optin = 0;
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  h->smem_optin = (size_t)optin;
  h->n = n;
  h->nnz = nnz;
  // forward view
  View &f = h->fwd;
  f.n = n; f.nnz = nnz;
  f.rp.assign(row_ptr, row_ptr + n + 1);
  f.ci.assign(col_idx, col_idx + nnz);
  f.diag = diag;
  // transposed view: counting sort by column; perm[q] = forward entry of q
  View &t = h->tr;
  t.n = n; t.nnz = nnz;
  t.rp.assign(n + 1, 0);
  t.ci.assign(nnz, 0);
  t.perm.assign(nnz, 0);
  t.diag.assign(n, -1);
  for (int k = 0; k < nnz; ++k) t.rp[col_idx[k] + 1]++;
  for (int j = 0; j < n; ++j) t.rp[j + 1] += t.rp[j];
  {
    std::vector<int> fill(t.rp.begin(), t.rp.end() - 1);
    for (int i = 0; i < n; ++i)
      for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
        const int q = fill[col_idx[k]]++;
        t.ci[q] = i;
        t.perm[q] = k;
        if (i == col_idx[k]) t.diag[col_idx[k]] = q;
      }
  }
  std::vector<int> row_of(nnz);
  for (int i = 0; i < n; ++i)
    for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) row_of[k] = i;
  if ((e = upload(&f.d_rp, f.rp)) != cudaSuccess ||
      (e = upload(&f.d_ci, f.ci)) != cudaSuccess ||
      (e = upload(&f.d_diag, f.diag)) != cudaSuccess ||
      (e = upload(&t.d_rp, t.rp)) != cudaSuccess ||
      (e = upload(&t.d_ci, t.ci)) != cudaSuccess ||
      (e = upload(&t.d_diag, t.diag)) != cudaSuccess ||
      (e = upload(&t.d_perm, t.perm)) != cudaSuccess ||
      (e = upload(&h->d_row_of, row_of)) != cudaSuccess ||
      (e = upload(&h->d_queue, std::vector<unsigned int>(2 * (1 + kHostSolveStreams) + kOrdWords,
                                                          0u))) != cudaSuccess) {
    free_view(h->fwd);
    free_view(h->tr);
    cudaFree(h->d_row_of);
    cudaFree(h->d_queue);
    delete h;
    return cuda_fail(e, "pattern upload");
  }
  *out = h;
  return CAMP_OK;
}

camp_status camp_solver_destroy(camp_solver_t h) {
  if (!h) return CAMP_OK;
  cudaSetDevice(h->device);
  cudaStreamSynchronize(h->stream);
  free_view(h->fwd);
  free_view(h->tr);
  for (auto &kv : h->mech.by_lanes) kv.second.release();
  cudaFree(h->d_row_of);
  cudaFree(h->d_queue);
  cudaFree(h->d_order_scratch);
  if (h->h_ord_err) cudaFreeHost(h->h_ord_err);
  if (h->h_hits) cudaFreeHost(h->h_hits);
  cudaFree(h->d_hits);
  cudaFree(h->d_ord);
  cudaFree(h->d_samp);
  if (h->ev_hits) cudaEventDestroy(h->ev_hits);
  cudaFree(h->h_dA); cudaFree(h->h_db); cudaFree(h->h_dx);
  cudaFree(h->h_dres); cudaFree(h->h_dit); cudaFree(h->h_dst);
  for (auto &s : h->h_streams) if (s) cudaStreamDestroy(s);
  for (auto &ev : h->h_in) if (ev) cudaEventDestroy(ev);
  for (auto &ev : h->h_done) if (ev) cudaEventDestroy(ev);
  if (h->h_start) cudaEventDestroy(h->h_start);
  delete h;
  return CAMP_OK;
}

camp_status camp_solver_set_stream(camp_solver_t h, void *stream) {
  if (!h) return fail(CAMP_EINVAL, "null solver handle");
  h->stream = (cudaStream_t)stream;
  return CAMP_OK;
}

camp_status camp_solver_set_arrangement(camp_solver_t h, int arrangement,
                                        int lanes_per_cell, int cells_per_block,
                                        int warps_per_block) {
  if (!h) return fail(CAMP_EINVAL, "null solver handle");
  if (arrangement == CAMP_ARR_AUTO) {
    h->arrangement = arrangement;
    h->wpb = warps_per_block > 0 ? warps_per_block : 0;
    return CAMP_OK;
  }
  if (arrangement == CAMP_ARR_WARP) {
    if (lanes_per_cell < 1 || lanes_per_cell > 32 || (lanes_per_cell & (lanes_per_cell - 1)))
      return fail(CAMP_EINVAL, "lanes_per_cell must be a power of two in [1, 32]");
    if ((h->n + lanes_per_cell - 1) / lanes_per_cell > kMaxE)
      return fail(CAMP_EUNSUPPORTED, "n=%d needs more than %d rows per lane at %d lanes",
                  h->n, kMaxE, lanes_per_cell);
    if (warps_per_block < 0 || warps_per_block > 8)
      return fail(CAMP_EINVAL, "warps_per_block must be in [0, 8]");
    h->arrangement = arrangement;
    h->lanes = lanes_per_cell;
    h->wpb = warps_per_block;
    return CAMP_OK;
  }
  if (arrangement == CAMP_ARR_BLOCK || arrangement == CAMP_ARR_BLOCK_COUPLED) {
    if (cells_per_block < 1 || cells_per_block * h->n > 1024)
      return fail(CAMP_EINVAL, "cells_per_block*n must be in [n, 1024]");
    h->arrangement = arrangement;
    h->cpb = cells_per_block;
    return CAMP_OK;
  }
  return fail(CAMP_EINVAL, "unknown arrangement %d", arrangement);
}

camp_status camp_solver_set_ordering(camp_solver_t h, int ordering) {
  if (!h) return fail(CAMP_EINVAL, "null solver handle");
  if (ordering < 0 || ordering > 2) return fail(CAMP_EINVAL, "ordering must be 0, 1 or 2");
  h->ordering = ordering;
  return CAMP_OK;
}

camp_status camp_solver_get_fault(camp_solver_t h, int *ordering_timed_out) {
  if (!h || !ordering_timed_out) return fail(CAMP_EINVAL, "null argument");
  *ordering_timed_out = 0;
  if (h->h_ord_err && *(volatile int *)h->h_ord_err) {
    *ordering_timed_out = 1;
    *(volatile int *)h->h_ord_err = 0;
  }
  return CAMP_OK;
}

camp_status camp_solver_set_single_tail(camp_solver_t h, int pairs) {
  if (!h) return fail(CAMP_EINVAL, "null solver handle");
  std::lock_guard<std::mutex> lock(h->mu);
  h->single_tail = pairs < 0 ? -1 : pairs;
  return CAMP_OK;
}

camp_status camp_solver_set_test_hooks(camp_solver_t h, long long ordering_wait_cycles,
                                       int refuse_cooperative) {
  if (!h) return fail(CAMP_EINVAL, "null solver handle");
  if (ordering_wait_cycles < 0) return fail(CAMP_EINVAL, "ordering_wait_cycles < 0");
  h->ord_wait = ordering_wait_cycles ? ordering_wait_cycles : kOrdWaitCycles;
  h->refuse_cooperative = refuse_cooperative ? 1 : 0;
  return CAMP_OK;
}

camp_status camp_solver_solve(camp_solver_t h, int cells, const double *A_vals,
                              const double *b, double *x, double tol,
                              int maxit, int *iters_out, double *resid_out) {
  return do_solve(h, cells, A_vals, b, x, tol, maxit, iters_out, resid_out,
                  nullptr, 0, h ? h->stream : nullptr, 0);
}

camp_status camp_solver_solve_ex(camp_solver_t h, int cells,
                                 const double *A_vals, const double *b,
                                 double *x, double tol, int maxit,
                                 int *iters_out, double *resid_out,
                                 int *status_out, int flags) {
  return do_solve(h, cells, A_vals, b, x, tol, maxit, iters_out, resid_out,
                  status_out, flags, h ? h->stream : nullptr, 0);
}

camp_status camp_solver_grad_A(camp_solver_t h, int cells,
                               const double *lambda, const double *x,
                               double *gA) {
  if (!h) return fail(CAMP_EINVAL, "null solver handle");
  if (cells < 0) return fail(CAMP_EINVAL, "cells < 0");
  if (cells == 0) return CAMP_OK;
  if (!lambda || !x || !gA) return fail(CAMP_EINVAL, "null array pointer");
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  GradArgs a;
  a.cells = cells; a.n = h->n; a.nnz = h->nnz;
  a.row_of = h->d_row_of; a.col_idx = h->fwd.d_ci;
  a.lambda = lambda; a.x = x; a.gA = gA;
  e = launch_grad(a, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "grad kernel launch");
  return CAMP_OK;
}

camp_status camp_solver_solve_host(camp_solver_t h, int cells,
                                   const double *A_vals, const double *b,
                                   double *x, double tol, int maxit,
                                   int *iters_out, double *resid_out,
                                   int *status_out) {
  if (!h) return fail(CAMP_EINVAL, "null solver handle");
  if (cells < 0) return fail(CAMP_EINVAL, "cells < 0");
  if (!(tol > 0.0) || !std::isfinite(tol)) return fail(CAMP_EINVAL, "tol must be finite and > 0");
  if (maxit < 1) return fail(CAMP_EINVAL, "maxit must be >= 1");
  if (cells == 0) return CAMP_OK;
  if (!A_vals || !b || !x || !iters_out || !resid_out)
    return fail(CAMP_EINVAL, "null array pointer");
  std::lock_guard<std::mutex> lock(h->mu);
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  const int n = h->n, nnz = h->nnz;
  if ((size_t)cells > h->h_cap_cells) {
    cudaFree(h->h_dA); cudaFree(h->h_db); cudaFree(h->h_dx);
    cudaFree(h->h_dres); cudaFree(h->h_dit); cudaFree(h->h_dst);
    h->h_dA = h->h_db = h->h_dx = h->h_dres = nullptr;
    h->h_dit = h->h_dst = nullptr;
    h->h_cap_cells = 0;
    if ((e = cudaMalloc(&h->h_dA, (size_t)cells * nnz * 8)) != cudaSuccess ||
        (e = cudaMalloc(&h->h_db, (size_t)cells * n * 8)) != cudaSuccess ||
        (e = cudaMalloc(&h->h_dx, (size_t)cells * n * 8)) != cudaSuccess ||
        (e = cudaMalloc(&h->h_dres, (size_t)cells * 8)) != cudaSuccess ||
        (e = cudaMalloc(&h->h_dit, (size_t)cells * 4)) != cudaSuccess ||
        (e = cudaMalloc(&h->h_dst, (size_t)cells * 4)) != cudaSuccess)
      return fail(CAMP_ENOMEM, "staging allocation: %s", cudaGetErrorString(e));
    h->h_cap_cells = (size_t)cells;
  }
  for (int q = 0; q < 2 + kHostSolveStreams; ++q)
    if (!h->h_streams[q] &&
        (e = cudaStreamCreateWithFlags(&h->h_streams[q], cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(e, "stream create");
  for (int q = 0; q < kHostChunks; ++q)
    if ((!h->h_in[q] && (e = cudaEventCreateWithFlags(&h->h_in[q], cudaEventDisableTiming)) != cudaSuccess) ||
        (!h->h_done[q] && (e = cudaEventCreateWithFlags(&h->h_done[q], cudaEventDisableTiming)) != cudaSuccess))
      return cuda_fail(e, "event create");
  cudaStream_t sin = h->h_streams[0], sout = h->h_streams[1];
  // order after earlier work on the handle's stream
  if (!h->h_start && (e = cudaEventCreateWithFlags(&h->h_start, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_fail(e, "event create");
  cudaEventRecord(h->h_start, h->stream);
  cudaStreamWaitEvent(sin, h->h_start, 0);
  // Pipeline: b in one copy, then A in chunks of shrinking size back to back
  // on the copy-in stream (few large copies keep the host link busy; a small
  // last chunk keeps the solve after the last byte short); each chunk's solve
  // starts on the next solve stream once its A has landed, so the solves of
  // consecutive chunks overlap.  The copies are enqueued first: the link
  // starts while the host sets up the rest.
  int nchunk = 1;
  while (nchunk < kHostChunks && cells >= (nchunk + 1) * 1024) ++nchunk;
  int c0s[kHostChunks + 1];
  {
    long tw = 0, acc = 0;
    for (int q = 0; q < nchunk; ++q) tw += nchunk + 2 - q;
    c0s[0] = 0;
    for (int q = 0; q < nchunk; ++q) {
      acc += nchunk + 2 - q;
      c0s[q + 1] = (int)((long)cells * acc / tw);
    }
    c0s[nchunk] = cells;
  }
  cudaMemcpyAsync(h->h_db, b, (size_t)cells * n * 8, cudaMemcpyHostToDevice, sin);
  // each copy ends at the first 4 KiB boundary of the source at or past its
  // chunk's last cell (a copy that starts inside a page ran 10-20 us slower
  // per boundary); a chunk's solve waits for the copy that holds its last byte
  {
    const size_t totA = (size_t)cells * nnz * 8;
    const uintptr_t base = reinterpret_cast<uintptr_t>(A_vals);
    size_t from = 0;
    for (int q = 0; q < nchunk; ++q) {
      const size_t want = (size_t)c0s[q + 1] * nnz * 8;
      const size_t to = q + 1 == nchunk
                            ? totA
                            : std::min(totA, (size_t)(((base + want + 4095) & ~(uintptr_t)4095) - base));
      if (to > from)
        cudaMemcpyAsync(reinterpret_cast<char *>(h->h_dA) + from,
                        reinterpret_cast<const char *>(A_vals) + from, to - from,
                        cudaMemcpyHostToDevice, sin);
      cudaEventRecord(h->h_in[q], sin);
      from = std::max(from, to);
    }
  }
  for (int q = 1; q < 2 + kHostSolveStreams; ++q) cudaStreamWaitEvent(h->h_streams[q], h->h_start, 0);
  // Outputs in host memory the device can address (pinned or mapped) are
  // written by the kernels directly; otherwise they are staged on the device
  // and copied back per chunk.
  auto device_view = [](const void *p) -> void * {
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return (pa.type == cudaMemoryTypeHost || pa.type == cudaMemoryTypeManaged) ? pa.devicePointer
                                                                               : nullptr;
  };
  double *dx = (double *)device_view(x);
  int *dit = (int *)device_view(iters_out);
  double *dres = (double *)device_view(resid_out);
  int *dst = status_out ? (int *)device_view(status_out) : nullptr;
  const bool direct = dx && dit && dres && (!status_out || dst);
  camp_status rs = CAMP_OK;
  for (int q = 0; q < nchunk; ++q) {
    const int c0 = c0s[q], cn = c0s[q + 1] - c0;
    if (cn <= 0) continue;
    cudaStream_t scomp = h->h_streams[2 + q % kHostSolveStreams];
    cudaStreamWaitEvent(scomp, h->h_in[q], 0);
    if (direct) {
      rs = do_solve(h, cn, h->h_dA + (size_t)c0 * nnz, h->h_db + (size_t)c0 * n,
                    dx + (size_t)c0 * n, tol, maxit, dit + c0, dres + c0,
                    dst ? dst + c0 : nullptr, 0, scomp, 1 + q % kHostSolveStreams);
      if (rs != CAMP_OK) break;
      cudaEventRecord(h->h_done[q], scomp);
      cudaStreamWaitEvent(sout, h->h_done[q], 0);
      continue;
    }
    rs = do_solve(h, cn, h->h_dA + (size_t)c0 * nnz, h->h_db + (size_t)c0 * n,
                  h->h_dx + (size_t)c0 * n, tol, maxit, h->h_dit + c0,
                  h->h_dres + c0, h->h_dst + c0, 0, scomp, 1 + q % kHostSolveStreams);
    if (rs != CAMP_OK) break;
    cudaEventRecord(h->h_done[q], scomp);
    cudaStreamWaitEvent(sout, h->h_done[q], 0);
    cudaMemcpyAsync(x + (size_t)c0 * n, h->h_dx + (size_t)c0 * n,
                    (size_t)cn * n * 8, cudaMemcpyDeviceToHost, sout);
    cudaMemcpyAsync(iters_out + c0, h->h_dit + c0, (size_t)cn * 4,
                    cudaMemcpyDeviceToHost, sout);
    cudaMemcpyAsync(resid_out + c0, h->h_dres + c0, (size_t)cn * 8,
                    cudaMemcpyDeviceToHost, sout);
    if (status_out)
      cudaMemcpyAsync(status_out + c0, h->h_dst + c0, (size_t)cn * 4,
                      cudaMemcpyDeviceToHost, sout);
  }
  // every stream's work precedes the copy-out stream's last wait or copy
  cudaError_t es = rs == CAMP_OK ? cudaStreamSynchronize(sout) : cudaSuccess;
  if (rs != CAMP_OK) {
    for (int q = 0; q < 2 + kHostSolveStreams; ++q) cudaStreamSynchronize(h->h_streams[q]);
    return rs;
  }
  if (es == cudaSuccess) es = cudaGetLastError();
  if (es != cudaSuccess) return cuda_fail(es, "solve_host");
  return CAMP_OK;
}

camp_status camp_solver_set_mechanism(camp_solver_t h, int R,
                                      const int *reactant_a,
                                      const int *reactant_b,
                                      const int *product,
                                      const double *rate_k) {
  if (!h) return fail(CAMP_EINVAL, "null solver handle");
  if (R < 0) return fail(CAMP_EINVAL, "R < 0");
  if (R > 0 && (!reactant_a || !reactant_b || !product || !rate_k))
    return fail(CAMP_EINVAL, "null mechanism array");
  const View &v = h->fwd;
  auto pos = [&](int i, int j) {
    for (int k = v.rp[i]; k < v.rp[i + 1]; ++k)
      if (v.ci[k] == j) return k;
    return -1;
  };
  Mechanism M;
  M.R = R;
  for (int r = 0; r < R; ++r) {
    const int a = reactant_a[r], b = reactant_b[r], c = product[r];
    const double k = rate_k[r];
    if (a < 0 || a >= v.n || c < 0 || c >= v.n || b >= v.n || b < -1)
      return fail(CAMP_EINVAL, "species index out of range in reaction %d", r);
    if (!std::isfinite(k)) return fail(CAMP_EINVAL, "rate constant of reaction %d is not finite", r);
    // (row, column, concentration factor, sign) of every Jacobian term
    int t[6][4];
    int nt = 0;
    if (b < 0) {
      int tt[2][4] = {{a, a, -1, -1}, {c, a, -1, 1}};
      for (int q = 0; q < 2; ++q) for (int z = 0; z < 4; ++z) t[q][z] = tt[q][z];
      nt = 2;
    } else {
      int tt[6][4] = {{a, a, b, -1}, {a, b, a, -1}, {b, a, b, -1},
                      {b, b, a, -1}, {c, a, b, 1},  {c, b, a, 1}};
      for (int q = 0; q < 6; ++q) for (int z = 0; z < 4; ++z) t[q][z] = tt[q][z];
      nt = 6;
    }
    for (int q = 0; q < nt; ++q) {
      const int e = pos(t[q][0], t[q][1]);
      if (e < 0)
        return fail(CAMP_EPATTERN, "reaction %d couples (%d, %d), which is not in the pattern",
                    r, t[q][0], t[q][1]);
      M.entry.push_back(e);
      M.spec.push_back(t[q][2]);
      M.val.push_back(t[q][3] * k);
    }
    // rate terms of f: the reaction's rate leaves a (and b), enters c
    const int rows[3] = {a, b, c};
    const double sg[3] = {-k, -k, k};
    for (int q = 0; q < 3; ++q) {
      if (rows[q] < 0) continue;
      M.rrow.push_back(rows[q]);
      M.ra.push_back(a);
      M.rb.push_back(b);
      M.rk.push_back(sg[q]);
    }
  }
  for (auto &kv : h->mech.by_lanes) kv.second.release();
  h->mech = std::move(M);
  return CAMP_OK;
}

namespace camp {
namespace {

// Per-lane term lists of the handle's mechanism for Lc lanes per cell, padded
// to the longest lane and laid out [term][lane]: the Jacobian terms of the
// lane's slots (tmeta = (species + 1) | slot row << 11) and the rate terms of
// the lane's rows (rmeta = (a + 1) | (b + 1) << 11 | e << 22, row sl + e Lc).
cudaError_t mech_terms(Mechanism &mech, int Lc, const Schedule &S, MechTerms **out) {
  auto it = mech.by_lanes.find(Lc);
  if (it != mech.by_lanes.end()) {
    *out = &it->second;
    return cudaSuccess;
  }
  auto pad = [Lc](std::vector<std::vector<std::pair<double, int>>> &lane,
                  std::vector<double> &val, std::vector<int> &meta) {
    size_t M = 1;
    for (auto &l : lane) M = std::max(M, l.size());
    val.assign(M * Lc, 0.0);
    meta.assign(M * Lc, 0);
    for (int q = 0; q < Lc; ++q)
      for (size_t p = 0; p < lane[q].size(); ++p) {
        val[p * Lc + q] = lane[q][p].first;
        meta[p * Lc + q] = lane[q][p].second;
      }
    return (int)M;
  };
  std::vector<std::vector<std::pair<double, int>>> lane(Lc), rlane(Lc);
  for (size_t q = 0; q < mech.entry.size(); ++q) {
    const int t = S.dst[mech.entry[q]];
    lane[t % Lc].push_back({mech.val[q], (mech.spec[q] + 1) | ((t / Lc) << 11)});
  }
  for (size_t q = 0; q < mech.rrow.size(); ++q) {
    const int row = mech.rrow[q];
    rlane[row % Lc].push_back(
        {mech.rk[q], (mech.ra[q] + 1) | ((mech.rb[q] + 1) << 11) | ((row / Lc) << 22)});
  }
  std::vector<double> tval, rval;
  std::vector<int> tmeta, rmeta;
  MechTerms T;
  T.count = pad(lane, tval, tmeta);
  T.rcount = pad(rlane, rval, rmeta);
  cudaError_t e;
  if ((e = upload(&T.d_tval, tval)) != cudaSuccess ||
      (e = upload(&T.d_tmeta, tmeta)) != cudaSuccess ||
      (e = upload(&T.d_rval, rval)) != cudaSuccess ||
      (e = upload(&T.d_rmeta, rmeta)) != cudaSuccess) {
    T.release();
    return e;
  }
  *out = &mech.by_lanes.emplace(Lc, T).first->second;
  return cudaSuccess;
}

}  // namespace
}  // namespace camp

// Launch arguments shared by the fused assembly and the Newton launches;
// extra_vectors = shared vectors per cell beyond the solve's own.  Returns CAMP_OK or the error.
static camp_status fused_args(camp_solver_t h, int cells, int extra_vectors, OccFn occ_fn,
                              WarpArgs *pa, int *pE, int *pwpb, size_t *psmem) {
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  View &v = h->fwd;
  const int Lc = (h->arrangement == CAMP_ARR_WARP) ? h->lanes : auto_lanes(v.n, kAutoRowsPerLane);
  const int E = Lc ? (v.n + Lc - 1) / Lc : 0;
  if (Lc == 0 || E > 8)
    return fail(CAMP_EUNSUPPORTED, "fused assembly supports at most 8 rows per lane (n=%d)", v.n);
  Schedule *S = nullptr;
  if ((e = view_schedule(v, Lc, &S)) != cudaSuccess) return cuda_fail(e, "schedule upload");
  if (S->L > 2047) return fail(CAMP_EUNSUPPORTED, "more than 2047 slots per lane");
  MechTerms *T = nullptr;
  if ((e = mech_terms(h->mech, Lc, *S, &T)) != cudaSuccess) return cuda_fail(e, "mechanism upload");
  int wpb = h->wpb > 0 ? h->wpb : 4;
  int segA = 0, segV = 0, segStride = 0;
  size_t smem = warp_smem(v, Lc, S->L, wpb, &segA, &segV, &segStride, extra_vectors);
  while (smem > h->smem_optin && wpb > 1)
    smem = warp_smem(v, Lc, S->L, --wpb, &segA, &segV, &segStride, extra_vectors);
  if (smem > h->smem_optin) return fail(CAMP_EUNSUPPORTED, "cell does not fit in shared memory");
  if (h->wpb == 0 &&
      (e = pick_warps_per_block(v, Lc, S->L, E, extra_vectors, h->smem_optin, occ_fn,
                                &S->auto_wpb[extra_vectors ? 2 : 1], &wpb, &smem, &segA, &segV,
                                &segStride)) != cudaSuccess)
    return cuda_fail(e, "occupancy");
  WarpArgs a = {};
  a.cells = cells; a.n = v.n; a.nnz = v.nnz;
  a.Lc = Lc; a.log2Lc = ilog2(Lc); a.k = 32 / Lc; a.L = S->L;
  a.segA = segA; a.segV = segV; a.segStride = segStride;
  a.ngroups = (cells + a.k - 1) / a.k;
  a.sched = S->d_words; a.src = S->d_src;
  a.dst = S->d_dst; a.padfrom = S->d_padfrom; a.dslot = S->d_dslot;
  a.x0_given = 0;
  a.queue = h->d_queue;
  a.tval = T->d_tval; a.tmeta = T->d_tmeta; a.tcount = T->count;
  a.rval = T->d_rval; a.rmeta = T->d_rmeta; a.rcount = T->rcount;
  *pa = a;
  *pE = E;
  *pwpb = wpb;
  *psmem = smem;
  return CAMP_OK;
}

camp_status camp_solver_assemble_solve(camp_solver_t h, int cells,
                                       const double *conc, const double *gamma,
                                       const double *b, double *x, double tol,
                                       int maxit, int *iters_out,
                                       double *resid_out, int *status_out) {
  if (!h) return fail(CAMP_EINVAL, "null solver handle");
  if (cells < 0) return fail(CAMP_EINVAL, "cells < 0");
  if (!(tol > 0.0) || !std::isfinite(tol)) return fail(CAMP_EINVAL, "tol must be finite and > 0");
  if (maxit < 1) return fail(CAMP_EINVAL, "maxit must be >= 1");
  if (cells == 0) return CAMP_OK;
  if (!conc || !gamma || !b || !x || !iters_out || !resid_out)
    return fail(CAMP_EINVAL, "null array pointer");
  WarpArgs a;
  int E = 0, wpb = 0;
  size_t smem = 0;
  camp_status rc = fused_args(h, cells, 0, assemble_occupancy, &a, &E, &wpb, &smem);
  if (rc != CAMP_OK) return rc;
  a.A = nullptr; a.b = b; a.x = x; a.iters = iters_out; a.resid = resid_out;
  a.status = status_out;
  a.tol = tol; a.maxit = maxit;
  a.conc = conc; a.gamma = gamma;
  int occ = 0;
  cudaError_t e;
  if ((e = assemble_occupancy(E, wpb, smem, &occ)) != cudaSuccess) return cuda_fail(e, "occupancy");
  if (occ < 1) occ = 1;
  const int grid = std::max(1, std::min((a.ngroups + wpb - 1) / wpb, h->sms * occ));
  rc = setup_gamma_ordering(h, a, smem - sched_smem_bytes(a.L * a.Lc), h->stream);
  if (rc != CAMP_OK) return rc;
  set_wave(a, grid, wpb);
  e = launch_cooperative(h, a.ord_ws != nullptr,
                         [&] { return launch_assemble(E, a, wpb, grid, smem, h->stream); });
  if (e == cudaErrorCooperativeLaunchTooLarge && a.ord_ws) {
    drop_gamma_ordering(a);
    e = launch_assemble(E, a, wpb, grid, smem, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(e, "assembly kernel launch");
  return CAMP_OK;
}

camp_status camp_solver_newton_solve(camp_solver_t h, int cells,
                                     const double *a_hist, const double *gamma,
                                     double *y, double newton_tol, int max_newton,
                                     double lin_tol, int lin_maxit,
                                     int *newton_iters_out, int *lin_iters_out,
                                     double *upd_out, double *resid_out,
                                     int *status_out) {
  if (!h) return fail(CAMP_EINVAL, "null solver handle");
  if (cells < 0) return fail(CAMP_EINVAL, "cells < 0");
  if (!(newton_tol > 0.0) || !std::isfinite(newton_tol))
    return fail(CAMP_EINVAL, "newton_tol must be finite and > 0");
  if (!(lin_tol > 0.0) || !std::isfinite(lin_tol))
    return fail(CAMP_EINVAL, "lin_tol must be finite and > 0");
  if (max_newton < 0) return fail(CAMP_EINVAL, "max_newton must be >= 0");
  if (lin_maxit < 1) return fail(CAMP_EINVAL, "lin_maxit must be >= 1");
  if (cells == 0) return CAMP_OK;
  if (!a_hist || !gamma || !y || !newton_iters_out || !lin_iters_out || !upd_out || !resid_out)
    return fail(CAMP_EINVAL, "null array pointer");
  WarpArgs a;
  int E = 0, wpb = 0;
  size_t smem = 0;
  camp_status rc = fused_args(h, cells, 1, newton_occupancy, &a, &E, &wpb, &smem);
  if (rc != CAMP_OK) return rc;
  a.A = nullptr; a.b = a_hist; a.x = y; a.iters = lin_iters_out; a.resid = resid_out;
  a.status = status_out;
  a.tol = lin_tol; a.maxit = lin_maxit;
  a.conc = nullptr; a.gamma = gamma;
  a.newton_tol = newton_tol; a.max_newton = max_newton;
  a.newton_iters = newton_iters_out; a.upd = upd_out;
  int occ = 0;
  cudaError_t e;
  if ((e = newton_occupancy(E, wpb, smem, &occ)) != cudaSuccess) return cuda_fail(e, "occupancy");
  if (occ < 1) occ = 1;
  const int grid = std::max(1, std::min((a.ngroups + wpb - 1) / wpb, h->sms * occ));
  rc = setup_gamma_ordering(h, a, smem - sched_smem_bytes(a.L * a.Lc), h->stream);
  if (rc != CAMP_OK) return rc;
  set_wave(a, grid, wpb);
  e = launch_cooperative(h, a.ord_ws != nullptr,
                         [&] { return launch_newton(E, a, wpb, grid, smem, h->stream); });
  if (e == cudaErrorCooperativeLaunchTooLarge && a.ord_ws) {
    drop_gamma_ordering(a);
    e = launch_newton(E, a, wpb, grid, smem, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(e, "Newton kernel launch");
  return CAMP_OK;
}

camp_status camp_solver_solve_mixed(camp_solver_t h, int cells,
                                    const double *A_vals, const double *b,
                                    double *x, double tol, int max_sweeps,
                                    double tol_inner, int maxit_inner,
                                    int *iters_out, int *sweeps_out,
                                    double *resid_out, int *status_out) {
  if (!h) return fail(CAMP_EINVAL, "null solver handle");
  if (cells < 0) return fail(CAMP_EINVAL, "cells < 0");
  if (!(tol > 0.0) || !std::isfinite(tol)) return fail(CAMP_EINVAL, "tol must be finite and > 0");
  if (!(tol_inner > 0.0) || !(tol_inner < 1.0)) return fail(CAMP_EINVAL, "tol_inner must be in (0, 1)");
  if (max_sweeps < 1 || maxit_inner < 1) return fail(CAMP_EINVAL, "max_sweeps and maxit_inner must be >= 1");
  if (cells == 0) return CAMP_OK;
  if (!A_vals || !b || !x || !iters_out || !resid_out)
    return fail(CAMP_EINVAL, "null array pointer");
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  View &v = h->fwd;
  int Lc = (h->arrangement == CAMP_ARR_WARP) ? h->lanes : auto_lanes(v.n, kAutoRowsPerLaneMixed);
  if (Lc == 0) return fail(CAMP_EUNSUPPORTED, "no warp arrangement fits n=%d", v.n);
  const int E = (v.n + Lc - 1) / Lc;
  if (E > kMaxE) return fail(CAMP_EUNSUPPORTED, "n=%d too large for %d lanes per cell", v.n, Lc);
  Schedule *S = nullptr;
  if ((e = view_schedule(v, Lc, &S)) != cudaSuccess) return cuda_fail(e, "schedule upload");
  // FP64 A in shared memory unless that costs resident warps (then the
  // outer residual product reads it through L1)
  const int wpb0 = h->wpb > 0 ? h->wpb : 4;
  int wpb = wpb0, segA = 0, segV = 0, best_warps = -1;
  bool a64 = true;
  size_t smem = 0;
  for (int s64 = 1; s64 >= 0; --s64) {
    int w = wpb0;
    size_t sm = mixed_smem(v, Lc, S->L, w, &segA, &segV, s64 != 0);
    while (sm > h->smem_optin && w > 1) sm = mixed_smem(v, Lc, S->L, --w, &segA, &segV, s64 != 0);
    if (sm > h->smem_optin) continue;
    int occ = 0;
    if ((e = mixed_occupancy(E, w, sm, &occ)) != cudaSuccess) return cuda_fail(e, "occupancy");
    if (occ * w > best_warps) {  // resident warps per SM; a tie keeps the staged FP64 A
      best_warps = occ * w;
      a64 = s64 != 0;
      wpb = w;
    }
  }
  if (best_warps < 0) return fail(CAMP_EUNSUPPORTED, "cell does not fit in shared memory");
  smem = mixed_smem(v, Lc, S->L, wpb, &segA, &segV, a64);
  MixedArgs a = {};
  a.cells = cells; a.n = v.n; a.nnz = v.nnz;
  a.Lc = Lc; a.log2Lc = ilog2(Lc); a.k = 32 / Lc; a.L = S->L;
  a.segA = segA; a.segV = segV; a.ngroups = (cells + a.k - 1) / a.k;
  a.A = A_vals; a.b = b; a.x = x; a.iters = iters_out; a.sweeps = sweeps_out;
  a.resid = resid_out; a.status = status_out; a.sched = S->d_words; a.src = S->d_src;
  a.dst = S->d_dst; a.padfrom = S->d_padfrom; a.dslot = S->d_dslot;
  a.tol = tol; a.max_sweeps = max_sweeps; a.tol_in = (float)tol_inner;
  a.maxit_in = maxit_inner;
  a.a64_smem = a64 ? 1 : 0;
  a.queue = h->d_queue;  // the handle's own stream: queue pair 0
  // Ordering pays here only by pairing: with one cell per warp (the automatic
  // choice above 48 species) its prologue costs more than hardest-first saves
  // (131 against 125 us at 80 species x 10,000 cells).
  bool calibrate = false;
  if (a.k > 1) {
    const camp_status rs = setup_ordering(h, a, A_vals, smem - sched_smem_bytes(S->L * Lc),
                                          h->stream, &calibrate);
    if (rs != CAMP_OK) return rs;
  }
  int occ = 0;
  if ((e = mixed_occupancy(E, wpb, smem, &occ)) != cudaSuccess) return cuda_fail(e, "occupancy");
  if (occ < 1) occ = 1;
  const int need = (a.ngroups + wpb - 1) / wpb;
  const int grid = std::max(1, std::min(need, h->sms * occ));
  set_wave(a, grid, wpb);
  e = launch_cooperative(h, a.ord_ws != nullptr,
                         [&] { return launch_mixed(E, a, wpb, grid, smem, h->stream); });
  if (e == cudaErrorCooperativeLaunchTooLarge && a.ord_ws) {
    const camp_status rs = fall_back_to_separate_ordering(h, a, A_vals, h->stream);
    if (rs != CAMP_OK) return rs;
    calibrate = false;
    e = launch_mixed(E, a, wpb, grid, smem, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(e, "mixed kernel launch");
  return calibrate ? read_back_hits(h, h->stream) : CAMP_OK;
}


// ---- persistent multi-mechanism batch ------------------------------------

struct camp_batch {
  int device = 0, sms = 0;
  size_t smem_optin = 0;
  int nmech = 0;
  camp_solver *mech[kMaxMech] = {};
  cudaStream_t stream = nullptr;
  int E = 0, wpb = 0, a_smem = 1;   // 0 = automatic
  unsigned int *d_counter = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t knode = nullptr;
  int g_E = 0, g_wpb = 0, g_asmem = -1, g_grid = 0;
  size_t g_smem = 0;
  // difficulty ordering (camp_batch_set_ordering, default on): per-cell
  // classes, the order and per-mechanism class counters, grown on demand;
  // the graph then starts with a memset, a classify and a scatter node
  int ordering = 1;
  unsigned char *d_ord = nullptr;
  size_t ord_cap = 0;  // cells
  cudaGraphNode_t cnode = nullptr, snode = nullptr;
  int g_ordered = -1, g_ogrid = 0, g_sgrid = 0;
  void *g_ordbuf = nullptr;
};

static void batch_drop_graph(camp_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->knode = nullptr;
  b->cnode = nullptr;
  b->snode = nullptr;
  b->g_asmem = -1;
  b->g_ordered = -1;
}

camp_status camp_batch_create(camp_batch_t *out, int nmech,
                              const camp_solver_t *mechs) {
  if (!out) return fail(CAMP_EINVAL, "null output handle pointer");
  *out = nullptr;
  if (nmech < 1 || nmech > kMaxMech)
    return fail(CAMP_EINVAL, "nmech=%d outside [1, %d]", nmech, kMaxMech);
  if (!mechs) return fail(CAMP_EINVAL, "null mechanism array");
  for (int m = 0; m < nmech; ++m)
    if (!mechs[m]) return fail(CAMP_EINVAL, "null solver handle for mechanism %d", m);
  camp_batch *b = new (std::nothrow) camp_batch();
  if (!b) return fail(CAMP_ENOMEM, "host allocation failed");
  b->nmech = nmech;
  for (int m = 0; m < nmech; ++m) b->mech[m] = mechs[m];
  b->device = mechs[0]->device;
  b->sms = mechs[0]->sms;
  b->smem_optin = mechs[0]->smem_optin;
  cudaError_t e = cudaSetDevice(b->device);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(unsigned int));
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "batch create");
  }
  *out = b;
  return CAMP_OK;
}

camp_status camp_batch_destroy(camp_batch_t b) {
  if (!b) return CAMP_OK;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  batch_drop_graph(b);
  cudaFree(b->d_counter);
  cudaFree(b->d_ord);
  delete b;
  return CAMP_OK;
}

camp_status camp_batch_set_stream(camp_batch_t b, void *stream) {
  if (!b) return fail(CAMP_EINVAL, "null batch handle");
  b->stream = (cudaStream_t)stream;
  return CAMP_OK;
}

camp_status camp_batch_set_config(camp_batch_t b, int rows_per_lane,
                                  int warps_per_block, int stage_A_in_smem) {
  if (!b) return fail(CAMP_EINVAL, "null batch handle");
  if (rows_per_lane != 0 && rows_per_lane != 3 && rows_per_lane != 4 &&
      rows_per_lane != 5 && rows_per_lane != 6 && rows_per_lane != 8)
    return fail(CAMP_EINVAL, "rows_per_lane must be 0 (auto), 3, 4, 5, 6 or 8");
  if (warps_per_block < 0 || warps_per_block > 8)
    return fail(CAMP_EINVAL, "warps_per_block must be in [0, 8]");
  b->E = rows_per_lane;
  b->wpb = warps_per_block;
  b->a_smem = stage_A_in_smem ? 1 : 0;
  return CAMP_OK;
}

camp_status camp_batch_set_ordering(camp_batch_t b, int ordering) {
  if (!b) return fail(CAMP_EINVAL, "null batch handle");
  if (ordering < 0 || ordering > 1) return fail(CAMP_EINVAL, "ordering must be 0 or 1");
  b->ordering = ordering;
  return CAMP_OK;
}

camp_status camp_batch_solve(camp_batch_t b, const int *cells,
                             const double *const *A_vals,
                             const double *const *bvec, double *const *x,
                             double tol, int maxit, int *const *iters_out,
                             double *const *resid_out, int *const *status_out) {
  if (!b) return fail(CAMP_EINVAL, "null batch handle");
  if (!cells || !A_vals || !bvec || !x || !iters_out || !resid_out)
    return fail(CAMP_EINVAL, "null argument array");
  if (!(tol > 0.0) || !std::isfinite(tol)) return fail(CAMP_EINVAL, "tol must be finite and > 0");
  if (maxit < 1) return fail(CAMP_EINVAL, "maxit must be >= 1");
  int max_n = 0;
  for (int m = 0; m < b->nmech; ++m) {
    if (cells[m] < 0) return fail(CAMP_EINVAL, "cells[%d] < 0", m);
    if (cells[m] > 0 && (!A_vals[m] || !bvec[m] || !x[m] || !iters_out[m] || !resid_out[m]))
      return fail(CAMP_EINVAL, "null array pointer for mechanism %d", m);
    max_n = std::max(max_n, b->mech[m]->n);
  }
  cudaError_t e = cudaSetDevice(b->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  // rows per lane shared by all mechanisms (one kernel instantiation)
  static const int kEs[] = {3, 4, 5, 6, 8};
  int E = b->E;
  if (E == 0) {
    E = 5;
    while ((max_n + 31) / 32 > E) E = (E == 5) ? 6 : 8;
  }
  if ((max_n + 31) / 32 > E)
    return fail(CAMP_EUNSUPPORTED, "n=%d needs more than %d rows per lane", max_n, E);
  (void)kEs;
  const bool asmem = b->a_smem != 0;
  // queue order: mechanisms with more species first
  int order[kMaxMech];
  for (int m = 0; m < b->nmech; ++m) order[m] = m;
  std::stable_sort(order, order + b->nmech,
                   [&](int p, int q) { return b->mech[p]->n > b->mech[q]->n; });
  BatchArgs args;
  memset(&args, 0, sizeof args);
  args.nmech = b->nmech;
  args.counter = b->d_counter;
  int items = 0, warp_doubles = 0;
  for (int q = 0; q < b->nmech; ++q) {
    const int m = order[q];
    camp_solver *h = b->mech[m];
    View &v = h->fwd;
    int Lc = 1;
    while ((v.n + Lc - 1) / Lc > E) Lc *= 2;
    Schedule *S = nullptr;
    if ((e = view_schedule(v, Lc, &S)) != cudaSuccess) return cuda_fail(e, "schedule upload");
    WarpArgs &a = args.m[q];
    a.cells = cells[m]; a.n = v.n; a.nnz = v.nnz;
    a.Lc = Lc; a.log2Lc = ilog2(Lc); a.k = 32 / Lc; a.L = S->L;
    a.segA = asmem ? ((S->L * Lc + 1) & ~1) : 0;
    a.segV = ((E * Lc + 1) + 1) & ~1;
    a.segStride = bank_spread_stride(a.segA + warp_vectors(E) * a.segV, a.k);
    a.ngroups = (cells[m] + a.k - 1) / a.k;
    a.A = A_vals[m]; a.b = bvec[m]; a.x = x[m]; a.iters = iters_out[m];
    a.resid = resid_out[m]; a.status = status_out ? status_out[m] : nullptr;
    a.sched = S->d_words; a.src = S->d_src; a.dslot = S->d_dslot;
    a.dst = S->d_dst; a.padfrom = S->d_padfrom;
    a.tol = tol; a.maxit = maxit; a.x0_given = 0; a.queue = nullptr;
    args.item_begin[q] = items;
    items += a.ngroups;
    warp_doubles = std::max(warp_doubles, a.k * a.segStride);
  }
  args.item_begin[b->nmech] = items;
  args.total_items = items;
  args.warp_doubles = warp_doubles;
  if (items == 0) return CAMP_OK;
  // hardest first within each mechanism (mechanisms stay largest first)
  BatchOrderArgs oa;
  memset(&oa, 0, sizeof oa);
  oa.nmech = b->nmech;
  for (int q = 0; q < b->nmech; ++q) {
    const int m = order[q];
    oa.A[q] = A_vals[m];
    oa.diag[q] = b->mech[m]->fwd.d_diag;
    oa.n[q] = b->mech[m]->n;
    oa.nnz[q] = b->mech[m]->nnz;
    oa.cell_begin[q + 1] = oa.cell_begin[q] + cells[m];
  }
  const int total_cells = oa.cell_begin[b->nmech];
  const bool ordered = b->ordering && total_cells > 1;
  const size_t cnt_bytes = (size_t)b->nmech * 2 * kOrdClasses * sizeof(int);
  if (ordered) {
    if ((size_t)total_cells > b->ord_cap) {
      cudaFree(b->d_ord);
      b->d_ord = nullptr;
      b->ord_cap = 0;
      // counters, the order (4 bytes per cell), then the classes (1 byte per cell)
      if ((e = cudaMalloc(&b->d_ord, cnt_bytes + (size_t)total_cells * 5)) != cudaSuccess)
        return fail(CAMP_ENOMEM, "batch ordering scratch: %s", cudaGetErrorString(e));
      b->ord_cap = (size_t)total_cells;
    }
    oa.counts = (int *)b->d_ord;
    oa.order = (int *)(b->d_ord + cnt_bytes);
    oa.cls = b->d_ord + cnt_bytes + b->ord_cap * 4;
    for (int q = 0; q < b->nmech; ++q) args.m[q].order = oa.order + oa.cell_begin[q];
  }
  const int ogrid = (int)std::max(1L, std::min(((long)total_cells * 32 + 255) / 256,
                                                (long)b->sms * 8));
  const int sgrid = (total_cells + 255) / 256;
  void *oparams[] = {&oa};
  int wpb = b->wpb > 0 ? b->wpb : 4;
  size_t smem = (size_t)wpb * warp_doubles * 8;
  while (smem > b->smem_optin && wpb > 1) smem = (size_t)(--wpb) * warp_doubles * 8;
  if (smem > b->smem_optin) return fail(CAMP_EUNSUPPORTED, "a warp's cells do not fit in shared memory");
  if (b->wpb == 0) {  // the most resident warps per SM, 4 unless another count fits more
    int best = -1;
    for (int w : {4, 8, 6, 5, 3, 2, 1}) {
      const size_t sm = (size_t)w * warp_doubles * 8;
      int o = 0;
      if (sm > b->smem_optin) continue;
      if ((e = batch_prepare(E, asmem, w, sm, &o)) != cudaSuccess) return cuda_fail(e, "batch occupancy");
      if (o * w > best) {
        best = o * w;
        wpb = w;
      }
    }
    smem = (size_t)wpb * warp_doubles * 8;
  }
  int occ = 0;
  if ((e = batch_prepare(E, asmem, wpb, smem, &occ)) != cudaSuccess) return cuda_fail(e, "batch occupancy");
  if (occ < 1) occ = 1;
  const int grid = std::max(1, std::min(b->sms * occ, (items + wpb - 1) / wpb));
  void *kparams[] = {&args};
  cudaKernelNodeParams kp;
  memset(&kp, 0, sizeof kp);
  kp.func = const_cast<void *>(batch_kernel(E, asmem));
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(wpb * 32);
  kp.sharedMemBytes = (unsigned)smem;
  kp.kernelParams = kparams;
  cudaKernelNodeParams cp, sp;
  memset(&cp, 0, sizeof cp);
  cp.func = const_cast<void *>(batch_classify_kernel_fn());
  cp.gridDim = dim3(ogrid);
  cp.blockDim = dim3(256);
  cp.kernelParams = oparams;
  sp = cp;
  sp.func = const_cast<void *>(batch_scatter_kernel_fn());
  sp.gridDim = dim3(sgrid);
  if (!b->exec || b->g_E != E || b->g_wpb != wpb || b->g_asmem != (int)asmem ||
      b->g_grid != grid || b->g_smem != smem || b->g_ordered != (int)ordered ||
      (ordered && (b->g_ordbuf != (void *)b->d_ord || b->g_ogrid != ogrid ||
                   b->g_sgrid != sgrid))) {
    batch_drop_graph(b);
    cudaGraphNode_t mnode, onode;
    cudaMemsetParams mp;
    memset(&mp, 0, sizeof mp);
    mp.dst = b->d_counter;
    mp.value = 0;
    mp.elementSize = sizeof(unsigned int);
    mp.width = 1;
    mp.height = 1;
    mp.pitch = sizeof(unsigned int);
    cudaMemsetParams op = mp;  // the ordering's class counters
    op.dst = b->d_ord;
    op.width = cnt_bytes / sizeof(unsigned int);
    op.pitch = cnt_bytes;
    cudaGraphNode_t deps[2];
    int ndeps = 0;
    if ((e = cudaGraphCreate(&b->graph, 0)) != cudaSuccess ||
        (e = cudaGraphAddMemsetNode(&mnode, b->graph, nullptr, 0, &mp)) != cudaSuccess) {
      batch_drop_graph(b);
      return cuda_fail(e, "batch graph build");
    }
    deps[ndeps++] = mnode;
    if (ordered &&
        ((e = cudaGraphAddMemsetNode(&onode, b->graph, nullptr, 0, &op)) != cudaSuccess ||
         (e = cudaGraphAddKernelNode(&b->cnode, b->graph, &onode, 1, &cp)) != cudaSuccess ||
         (e = cudaGraphAddKernelNode(&b->snode, b->graph, &b->cnode, 1, &sp)) != cudaSuccess)) {
      batch_drop_graph(b);
      return cuda_fail(e, "batch graph build (ordering)");
    }
    if (ordered) deps[ndeps++] = b->snode;
    if ((e = cudaGraphAddKernelNode(&b->knode, b->graph, deps, ndeps, &kp)) != cudaSuccess ||
        (e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess) {
      batch_drop_graph(b);
      return cuda_fail(e, "batch graph build");
    }
    b->g_E = E; b->g_wpb = wpb; b->g_asmem = asmem; b->g_grid = grid; b->g_smem = smem;
    b->g_ordered = ordered ? 1 : 0;
    b->g_ordbuf = b->d_ord;
    b->g_ogrid = ogrid;
    b->g_sgrid = sgrid;
  } else {
    if ((e = cudaGraphExecKernelNodeSetParams(b->exec, b->knode, &kp)) != cudaSuccess ||
        (ordered && ((e = cudaGraphExecKernelNodeSetParams(b->exec, b->cnode, &cp)) != cudaSuccess ||
                     (e = cudaGraphExecKernelNodeSetParams(b->exec, b->snode, &sp)) != cudaSuccess)))
      return cuda_fail(e, "batch graph update");
  }
  if ((e = cudaGraphLaunch(b->exec, b->stream)) != cudaSuccess)
    return cuda_fail(e, "batch graph launch");
  return CAMP_OK;
}


// ---- solve without any device allocation -------------------------------
//
// For callers that cannot call cudaMalloc: a host model that owns all device
// memory through its own pool, or a time loop that must not allocate once it
// runs.  camp_solve_noalloc needs no solver handle: the SpMV schedule and the
// diagonal positions, which camp_solver_create keeps in device memory of its
// own, are staged instead in the file-scope array below (kNoAllocScratchBytes,
// held by every GPU that loads the library until the process exits), and the
// plain warp kernel reads them from there.

}  // extern "C"

namespace camp {
namespace {
constexpr size_t kNoAllocScratchBytes = 256 * 1024;
constexpr int kNoAllocMaxDevices = 64;
}  // namespace
}  // namespace camp

static __device__ __align__(256) unsigned char g_noalloc_scratch[camp::kNoAllocScratchBytes];

namespace camp {
namespace {

std::mutex g_noalloc_mu;                              // guards the host buffers below
void *g_noalloc_dev[kNoAllocMaxDevices];              // device address of the scratch
SchedWord g_noalloc_words[kNoAllocScratchBytes / sizeof(SchedWord)];
int g_noalloc_dst[kNoAllocScratchBytes / sizeof(int)];
int g_noalloc_padfrom[32];
int g_noalloc_entry[kNoAllocScratchBytes / sizeof(SchedWord)];
int g_noalloc_order[1024], g_noalloc_diag[1024], g_noalloc_dslot[1024];
int g_noalloc_bin_rows[32][1024], g_noalloc_bin_count[32];
int g_noalloc_rem[32][1024], g_noalloc_rem_count[32], g_noalloc_cursor[32], g_noalloc_cur_row[32];
long g_noalloc_load[32];

// Same schedule as build_schedule (sched::build, with the static host
// buffers as its work space), written into the static host buffers (slot
// words, slot of every entry, first padding slot of every lane, slot of
// every diagonal); returns slots per lane or -1 if it needs more than
// cap_slots slots.
int noalloc_schedule(int n, const int *rp, const int *ci, int Lc, size_t cap_slots) {
  const sched::Work w = {g_noalloc_order, g_noalloc_load, &g_noalloc_bin_rows[0][0],
                         g_noalloc_bin_count, g_noalloc_cursor, g_noalloc_cur_row,
                         &g_noalloc_rem[0][0], g_noalloc_rem_count};
  const size_t cap = std::min(cap_slots, sizeof(g_noalloc_words) / sizeof(g_noalloc_words[0]));
  const int L = sched::build(n, rp, ci, g_noalloc_diag, Lc, cap, w, g_noalloc_words,
                             g_noalloc_entry, g_noalloc_dslot, g_noalloc_padfrom);
  if (L < 0) return -1;
  for (long t = 0; t < (long)L * Lc; ++t)
    if (g_noalloc_entry[t] >= 0) g_noalloc_dst[g_noalloc_entry[t]] = (int)t;
  return L;
}

}  // namespace
}  // namespace camp

extern "C" {

camp_status camp_solve_noalloc(int n, int nnz, const int *row_ptr,
                               const int *col_idx, int cells,
                               const double *A_vals, const double *b,
                               double *x, double tol, int maxit,
                               int *iters_out, double *resid_out,
                               int *status_out, void *stream) {
  if (!row_ptr || !col_idx) return fail(CAMP_EINVAL, "null pattern array");
  if (n < 1 || n > 1024) return fail(CAMP_EINVAL, "n=%d outside [1, 1024]", n);
  if (nnz < n || nnz > 65535) return fail(CAMP_EINVAL, "nnz=%d outside [n, 65535]", nnz);
  if (cells < 0) return fail(CAMP_EINVAL, "cells < 0");
  if (!(tol > 0.0) || !std::isfinite(tol)) return fail(CAMP_EINVAL, "tol must be finite and > 0");
  if (maxit < 1) return fail(CAMP_EINVAL, "maxit must be >= 1");
  if (row_ptr[0] != 0 || row_ptr[n] != nnz)
    return fail(CAMP_EPATTERN, "row_ptr[0] must be 0 and row_ptr[n] must equal nnz");
  const int Lc = auto_lanes(n, kAutoRowsPerLane);
  const int E = Lc ? (n + Lc - 1) / Lc : 0;
  if (Lc == 0 || E > kMaxE)
    return fail(CAMP_EUNSUPPORTED, "n=%d is too large for the warp kernel (at most %d)", n, 32 * kMaxE);
  if (cells > 0 && (!A_vals || !b || !x || !iters_out || !resid_out))
    return fail(CAMP_EINVAL, "null array pointer");

  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  for (int i = 0; i < n; ++i) {
    g_noalloc_diag[i] = -1;
    if (row_ptr[i + 1] < row_ptr[i]) return fail(CAMP_EPATTERN, "row_ptr decreases at row %d", i);
    if (row_ptr[i + 1] > nnz) return fail(CAMP_EPATTERN, "row_ptr[%d] exceeds nnz", i + 1);
    for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      const int j = col_idx[k];
      if (j < 0 || j >= n) return fail(CAMP_EPATTERN, "column %d out of range at entry %d", j, k);
      if (k > row_ptr[i] && j <= col_idx[k - 1])
        return fail(CAMP_EPATTERN, "columns not strictly increasing in row %d", i);
      if (j == i) g_noalloc_diag[i] = k;
    }
    if (g_noalloc_diag[i] < 0) return fail(CAMP_EPATTERN, "diagonal entry missing in row %d", i);
  }
  // scratch layout, 16-byte aligned pieces: [diagonal slots, n ints]
  // [first padding slot per lane, 32 ints][slot of every entry, nnz ints]
  // [slot words, L*Lc]
  const size_t diag_bytes = ((size_t)n * sizeof(int) + 15) & ~(size_t)15;
  const size_t pad_bytes = 32 * sizeof(int);
  const size_t dst_bytes = ((size_t)nnz * sizeof(int) + 15) & ~(size_t)15;
  const size_t head_bytes = diag_bytes + pad_bytes + dst_bytes;
  const size_t cap_slots = head_bytes < kNoAllocScratchBytes
                               ? (kNoAllocScratchBytes - head_bytes) / sizeof(SchedWord)
                               : 0;
  const int L = noalloc_schedule(n, row_ptr, col_idx, Lc, cap_slots);
  if (L < 0)
    return fail(CAMP_EUNSUPPORTED,
                "pattern needs more than the %zu-byte static scratch of camp_solve_noalloc "
                "(schedule %d lanes x slots plus %d diagonal positions); use a solver handle",
                kNoAllocScratchBytes, Lc, n);
  if (cells == 0) return CAMP_OK;

  cudaStream_t st = (cudaStream_t)stream;
  // a captured copy would read the host buffers above at replay time, after
  // later calls may have overwritten them
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
  if (cap != cudaStreamCaptureStatusNone)
    return fail(CAMP_EUNSUPPORTED, "camp_solve_noalloc does not run while its stream is capturing");
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(CAMP_EUNSUPPORTED, "device ordinal %d", dev);
  if (!g_noalloc_dev[dev]) {  // set-up, once per device, with that device current
    void *p = nullptr;
    if ((e = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess)
      return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
    g_noalloc_dev[dev] = p;
  }
  unsigned char *scratch = (unsigned char *)g_noalloc_dev[dev];
  int sms = 0, optin = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);

  WarpArgs a = {};
  a.cells = cells; a.n = n; a.nnz = nnz;
  a.Lc = Lc; a.log2Lc = ilog2(Lc); a.k = 32 / Lc; a.L = L;
  a.segA = (L * Lc + 1) & ~1;
  a.segV = ((E * Lc + 1) + 1) & ~1;
  a.segStride = bank_spread_stride(a.segA + warp_vectors(E) * a.segV, a.k);
  a.ngroups = (cells + a.k - 1) / a.k;
  a.A = A_vals; a.b = b; a.x = x; a.iters = iters_out; a.resid = resid_out;
  a.status = status_out;
  a.dslot = (const int *)scratch;
  a.padfrom = (const int *)(scratch + diag_bytes);
  a.dst = (const int *)(scratch + diag_bytes + pad_bytes);
  a.sched = (const SchedWord *)(scratch + head_bytes);
  a.src = nullptr;  // only the global-memory A path reads it
  a.tol = tol; a.maxit = maxit; a.x0_given = 0; a.queue = nullptr;
  int wpb = 4;
  const size_t sch = sched_smem_bytes(L * Lc);
  size_t smem = sch + (size_t)wpb * a.k * a.segStride * 8;
  while (smem > (size_t)optin && wpb > 1) smem = sch + (size_t)(--wpb) * a.k * a.segStride * 8;
  if (smem > (size_t)optin) return fail(CAMP_EUNSUPPORTED, "cell does not fit in shared memory");
  int occ = 0;
  if ((e = warp_occupancy(E, wpb, smem, &occ)) != cudaSuccess) return cuda_fail(e, "occupancy");
  if (occ < 1) occ = 1;
  const int grid = std::max(1, std::min((a.ngroups + wpb - 1) / wpb, sms * occ));
  // stage the schedule pieces (pageable source: each call returns once its
  // host buffer has been consumed)
  if ((e = cudaMemcpyAsync(scratch, g_noalloc_dslot, (size_t)n * sizeof(int),
                           cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(scratch + diag_bytes, g_noalloc_padfrom, (size_t)Lc * sizeof(int),
                           cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(scratch + diag_bytes + pad_bytes, g_noalloc_dst,
                           (size_t)nnz * sizeof(int), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(scratch + head_bytes, g_noalloc_words,
                           (size_t)L * Lc * sizeof(SchedWord), cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_fail(e, "staging into the static scratch");
  if ((e = launch_warp(E, a, wpb, grid, smem, st)) != cudaSuccess)
    return cuda_fail(e, "warp kernel launch");
  return CAMP_OK;
}

}  // extern "C"
