// Host-side construction of the warp kernels' static SpMV schedule, shared by
// the solver handle and the allocation-free entry point (it allocates
// nothing: every buffer is the caller's).
//
// One cell's product y = A v is split over the Lc lanes of its warp segment:
// whole rows are assigned to lanes by longest-processing-time-first bin
// packing (so every lane runs about nnz/Lc slots), each lane takes its rows
// in ascending order, and within a row the entries may come in any order.
// That last freedom is used to keep the shared-memory gather of v free of
// bank conflicts: in slot j every lane reads v[col] of the entry it takes,
// and a warp's 8-byte shared-memory access is served 16 lanes (128 bytes,
// 16 bank pairs) at a time.  The kernels place consecutive cells of a warp
// Lc doubles apart modulo 16 (bank pairs), so for a group of G = min(Lc, 16)
// lanes the reads of every cell in a half-warp fall on distinct bank pairs
// exactly when the columns the G lanes take have distinct residues modulo G
// (lanes that take the same column read one address, a broadcast).  For
// every slot and group the lanes are matched to residues by augmenting paths
// (Kuhn's algorithm, lanes with the fewest options first); a lane left
// unmatched takes a column another lane of its group already takes, if its
// row has one, else its first remaining entry.  With Lc = 32 the second
// half-warp is matched to the residues modulo 32 the first did not take, so
// a 4-byte access of all 32 lanes (the FP32 refinement kernel) is also
// conflict-free.
#pragma once
#include <stddef.h>

namespace camp {
namespace sched {

// Work buffers of build (caller-owned; sizes in elements).
struct Work {
  int *order;      // [n]
  long *load;      // [Lc]
  int *bin_rows;   // [Lc * n]
  int *bin_count;  // [Lc]
  int *cursor;     // [Lc] next row of the lane's list
  int *cur_row;    // [Lc] row in progress (-1: none)
  int *rem;        // [Lc * n] remaining entries (CSR positions) of the row in progress
  int *rem_count;  // [Lc]
};

// Kuhn's augmenting path: try to give lane q (index into the group) one of
// its residues; owner[r] is the lane holding residue r or -1.
inline bool augment(int q, const unsigned *opts, int *owner, unsigned *seen, int G) {
  for (int r = 0; r < G; ++r) {
    if (!((opts[q] >> r) & 1u) || ((*seen >> r) & 1u)) continue;
    *seen |= 1u << r;
    if (owner[r] < 0 || augment(owner[r], opts, owner, seen, G)) {
      owner[r] = q;
      return true;
    }
  }
  return false;
}

// Modelled shared-memory wavefronts of slot j's gathers beyond the ideal:
// for every group of G lanes (a half-warp's worth), the largest number of
// distinct columns sharing a residue modulo G, minus one; with Lc = 32 also
// the 4-byte access of all 32 lanes (residues modulo 32).  Padding lanes
// (entry -1) are left out: their column is set to a broadcast at the end.
inline int slot_cost(long j, int Lc, const unsigned *word, const int *entry) {
  const int G = Lc < 16 ? Lc : 16;
  int cost = 0;
  for (int pass = 0; pass < (Lc == 32 ? 2 : 1); ++pass) {
    const int M = pass ? 32 : G;          // residues
    const int span = pass ? 32 : G;       // lanes counted together
    for (int g0 = 0; g0 < Lc; g0 += span) {
      int cols[32], ncol = 0, cnt[32];
      for (int r = 0; r < M; ++r) cnt[r] = 0;
      for (int x = 0; x < span; ++x) {
        const size_t t = (size_t)j * Lc + g0 + x;
        if (entry[t] < 0) continue;
        const int c = (int)(word[t] & 0x7ffu);
        bool dup = false;
        for (int y = 0; y < ncol && !dup; ++y) dup = cols[y] == c;
        if (dup) continue;
        cols[ncol++] = c;
        ++cnt[c % M];
      }
      int worst = 0;
      for (int r = 0; r < M; ++r) worst = cnt[r] > worst ? cnt[r] : worst;
      cost += worst > 1 ? worst - 1 : 0;
    }
  }
  return cost;
}

// Exchange the entries of slots (ja, q) and (jb, q), two slots of one row
// of lane q; the row's end flag stays on its last slot.
inline void swap_slots(long ja, long jb, int q, int Lc, unsigned *word, int *entry) {
  const size_t ta = (size_t)ja * Lc + q, tb = (size_t)jb * Lc + q;
  const unsigned ea = word[ta] & 0x80000000u, eb = word[tb] & 0x80000000u;
  const unsigned wa = word[ta] & 0x7fffffffu, wb = word[tb] & 0x7fffffffu;
  word[ta] = wb | ea;
  word[tb] = wa | eb;
  const int k = entry[ta];
  entry[ta] = entry[tb];
  entry[tb] = k;
}

// Build the schedule of one orientation of the pattern (CSR rp, ci over n
// rows; diag[r] the CSR position of row r's diagonal entry).  Outputs, for
// slot t = j * Lc + q (lane q, slot j): word[t] = column | row << 11 | end of
// row << 31 and entry[t] = the CSR position it multiplies (padding: entry -1,
// no row end, and a column another lane of the group reads, so that the
// padding lane's read is a broadcast); dslot[r] = the slot of row r's
// diagonal entry;
// padfrom[q] = the lane's first padding slot.  Returns the slots per lane
// L, or -1 if L * Lc would exceed cap_slots (nothing past it is written).
inline int build(int n, const int *rp, const int *ci, const int *diag, int Lc, size_t cap_slots,
                 const Work &w, unsigned *word, int *entry, int *dslot, int *padfrom) {
  // rows, longest first (stable), onto the least-loaded lane (lowest on ties)
  for (int i = 0; i < n; ++i) w.order[i] = i;
  for (int i = 1; i < n; ++i) {
    const int r = w.order[i];
    const int len = rp[r + 1] - rp[r];
    int j = i - 1;
    while (j >= 0 && rp[w.order[j] + 1] - rp[w.order[j]] < len) {
      w.order[j + 1] = w.order[j];
      --j;
    }
    w.order[j + 1] = r;
  }
  for (int q = 0; q < Lc; ++q) {
    w.load[q] = 0;
    w.bin_count[q] = 0;
  }
  for (int i = 0; i < n; ++i) {
    const int r = w.order[i];
    int best = 0;
    for (int q = 1; q < Lc; ++q)
      if (w.load[q] < w.load[best]) best = q;
    w.load[best] += rp[r + 1] - rp[r];
    w.bin_rows[(size_t)best * n + w.bin_count[best]++] = r;
  }
  long L = 0;
  for (int q = 0; q < Lc; ++q) L = w.load[q] > L ? w.load[q] : L;
  if ((size_t)L * Lc > cap_slots) return -1;
  for (int q = 0; q < Lc; ++q) {  // ascending rows within a lane
    int *rows = w.bin_rows + (size_t)q * n;
    for (int i = 1; i < w.bin_count[q]; ++i) {
      const int r = rows[i];
      int j = i - 1;
      while (j >= 0 && rows[j] > r) {
        rows[j + 1] = rows[j];
        --j;
      }
      rows[j + 1] = r;
    }
    padfrom[q] = (int)w.load[q];
    w.cursor[q] = 0;
    w.cur_row[q] = -1;
    w.rem_count[q] = 0;
  }
  const int G = Lc < 16 ? Lc : 16;   // lanes matched together
  const int R = Lc < 32 ? G : 32;    // residues of the column taken
  int taken32[16];                   // residue mod 32 the first half took, per class mod 16
  for (long j = 0; j < L; ++j) {
    for (int q = 0; q < Lc; ++q) {   // lanes whose row is done move to the next one
      if (w.rem_count[q] > 0 || w.cursor[q] >= w.bin_count[q]) continue;
      const int r = w.bin_rows[(size_t)q * n + w.cursor[q]++];
      w.cur_row[q] = r;
      int *rem = w.rem + (size_t)q * n;
      for (int k = rp[r]; k < rp[r + 1]; ++k) rem[w.rem_count[q]++] = k;
    }
    for (int c = 0; c < 16; ++c) taken32[c] = -1;
    for (int g0 = 0; g0 < Lc; g0 += G) {
      unsigned opts[16];
      int owner[16], lane_of[16], pick[16];
      for (int x = 0; x < G; ++x) {
        opts[x] = 0u;
        owner[x] = -1;
        pick[x] = -1;
        const int q = g0 + x;
        const int *rem = w.rem + (size_t)q * n;
        for (int y = 0; y < w.rem_count[q]; ++y) {
          const int col = ci[rem[y]];
          const int cls = col % G;
          if (R == 32 && g0 > 0 && taken32[cls] >= 0 && col % 32 == taken32[cls]) continue;
          opts[x] |= 1u << cls;
        }
      }
      // lanes with the fewest options first
      for (int x = 0; x < G; ++x) lane_of[x] = x;
      for (int x = 1; x < G; ++x) {
        const int v = lane_of[x];
        const int pv = __builtin_popcount(opts[v]);
        int y = x - 1;
        while (y >= 0 && __builtin_popcount(opts[lane_of[y]]) > pv) {
          lane_of[y + 1] = lane_of[y];
          --y;
        }
        lane_of[y + 1] = v;
      }
      for (int x = 0; x < G; ++x) {
        unsigned seen = 0u;
        if (opts[lane_of[x]]) augment(lane_of[x], opts, owner, &seen, G);
      }
      // matched lanes: their first remaining entry of the residue
      for (int cls = 0; cls < G; ++cls) {
        const int x = owner[cls];
        if (x < 0) continue;
        const int q = g0 + x;
        const int *rem = w.rem + (size_t)q * n;
        for (int y = 0; y < w.rem_count[q]; ++y) {
          const int col = ci[rem[y]];
          if (col % G != cls) continue;
          if (R == 32 && g0 > 0 && taken32[cls] >= 0 && col % 32 == taken32[cls]) continue;
          pick[x] = y;
          break;
        }
      }
      // the others: a column a matched lane of the group takes (one address,
      // a broadcast), else the first remaining entry
      int first_col = -1;
      for (int x = 0; x < G; ++x)
        if (pick[x] >= 0) {
          const int *rx = w.rem + (size_t)(g0 + x) * n;
          if (first_col < 0) first_col = ci[rx[pick[x]]];
        }
      for (int x = 0; x < G; ++x) {
        const int q = g0 + x;
        if (pick[x] >= 0 || w.rem_count[q] == 0) continue;
        const int *rem = w.rem + (size_t)q * n;
        int found = -1;
        for (int y = 0; y < w.rem_count[q] && found < 0; ++y)
          for (int z = 0; z < G; ++z) {
            if (z == x || pick[z] < 0 || owner[ci[w.rem[(size_t)(g0 + z) * n + pick[z]]] % G] != z)
              continue;
            if (ci[w.rem[(size_t)(g0 + z) * n + pick[z]]] == ci[rem[y]]) {
              found = y;
              break;
            }
          }
        pick[x] = found >= 0 ? found : 0;
      }
      for (int x = 0; x < G; ++x) {
        const int q = g0 + x;
        const size_t t = (size_t)j * Lc + q;
        if (pick[x] < 0) {
          // padding: A = 0 and no row end; read a column another lane reads
          word[t] = first_col >= 0 ? (unsigned)first_col : 0u;
          entry[t] = -1;
          continue;
        }
        int *rem = w.rem + (size_t)q * n;
        const int k = rem[pick[x]];
        rem[pick[x]] = rem[--w.rem_count[q]];  // order of the rest does not matter
        const int r = w.cur_row[q];
        const int col = ci[k];
        word[t] = (unsigned)col | ((unsigned)r << 11) |
                  (w.rem_count[q] == 0 ? 0x80000000u : 0u);
        entry[t] = k;
        if (k == diag[r]) dslot[r] = (int)t;
        if (R == 32 && g0 == 0) taken32[col % 16] = col % 32;
      }
    }
  }
  // Local search: within each row, exchange the slots of two entries while
  // that lowers the modelled conflicts of the two slots (deterministic,
  // first improvement, at most 8 sweeps).
  for (int sweep = 0; sweep < 8; ++sweep) {
    bool improved = false;
    for (int q = 0; q < Lc; ++q) {
      long j0 = 0;
      while (j0 < w.load[q]) {
        long j1 = j0;  // the row's span [j0, j1]
        while (!(word[(size_t)j1 * Lc + q] & 0x80000000u)) ++j1;
        for (long ja = j0; ja < j1; ++ja)
          for (long jb = ja + 1; jb <= j1; ++jb) {
            const int before = slot_cost(ja, Lc, word, entry) + slot_cost(jb, Lc, word, entry);
            swap_slots(ja, jb, q, Lc, word, entry);
            const int after = slot_cost(ja, Lc, word, entry) + slot_cost(jb, Lc, word, entry);
            if (after < before) {
              improved = true;
            } else {
              swap_slots(ja, jb, q, Lc, word, entry);
            }
          }
        j0 = j1 + 1;
      }
    }
    if (!improved) break;
  }
  // diagonal slots and broadcast columns for the padding lanes
  for (long j = 0; j < L; ++j) {
    for (int g0 = 0; g0 < Lc; g0 += G) {
      int any = -1;
      for (int x = 0; x < G && any < 0; ++x)
        if (entry[(size_t)j * Lc + g0 + x] >= 0) any = (int)(word[(size_t)j * Lc + g0 + x] & 0x7ffu);
      for (int x = 0; x < G; ++x) {
        const size_t t = (size_t)j * Lc + g0 + x;
        if (entry[t] < 0) {
          word[t] = any >= 0 ? (unsigned)any : 0u;
          continue;
        }
        const int r = (int)((word[t] >> 11) & 0x7ffu);
        if (entry[t] == diag[r]) dslot[r] = (int)t;
      }
    }
  }
  return (int)L;
}

}  // namespace sched
}  // namespace camp
