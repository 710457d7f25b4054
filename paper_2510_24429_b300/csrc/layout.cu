// Device construction of the matrix layouts (Hyb) of one LP or of a batch of
// LPs stacked block-diagonally: row lengths, the renumbering of rows and
// columns by decreasing length, the transpose, and the packing of the rows
// into long-row units and slices. All of it is integer work and data
// movement, done once per context; the unit tables themselves (a few bytes
// per 32 rows) are computed on the host from the sorted row lengths. The
// layout is this engine's own; the paper only states A as a sparse matrix of
// its LP (Section 2).
//
// Orders are deterministic: the renumbering is a stable sort (rows of equal
// length keep their order), and every row of the transpose lists its entries
// in the order of the caller's rows, so two builds of the same LP are
// bit-identical.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace pdhg {
namespace {

constexpr int LT_TPB = 256;  // elementwise and warp-per-row kernels
constexpr int RS_TPB = 256;  // radix sort: one thread per digit value
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_TPB * RS_ITEMS;  // keys per block and pass
constexpr int SC_TPB = 256, SC_ITEMS = 8;
constexpr int SC_TILE = SC_TPB * SC_ITEMS;  // elements per block of the scan

int grid_of(long long threads) {
  const long long g = (threads + LT_TPB - 1) / LT_TPB;
  return (int)std::max(1LL, std::min(g, 148LL * 64));
}

__device__ __forceinline__ long long gtid() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long gstride() { return (long long)gridDim.x * blockDim.x; }

// ---- instance maps, lengths --------------------------------------------------

// out[i] = the instance owning element i: off[inst] <= i < off[inst + 1]
__global__ void k_instance_of(const int* __restrict__ off, int count, long long len, int* __restrict__ out) {
  for (long long i = gtid(); i < len; i += gstride()) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (off[mid] <= i)
        lo = mid;
      else
        hi = mid - 1;
    }
    out[i] = lo;
  }
}

// Global block-diagonal CSR from the instances' own arrays: row g of instance
// inst is its local row r = g - yoff[inst]; its entries get the global column
// xoff[inst] + local column, and rowid records their global row.
__global__ void k_globalize(const long long* __restrict__ lrp, const int* __restrict__ lci,
                            const long long* __restrict__ rpoff, const long long* __restrict__ zoff,
                            const int* __restrict__ xoff, const int* __restrict__ yoff, const int* __restrict__ rinst,
                            long long M, long long Z, long long* __restrict__ grp, int* __restrict__ gci,
                            int* __restrict__ rowid) {
  const int lane = threadIdx.x & 31;
  const long long w0 = gtid() >> 5, nw = gstride() >> 5;
  for (long long g = w0; g < M; g += nw) {
    const int inst = rinst ? rinst[g] : 0;
    const long long r = g - yoff[inst];
    const long long* rp = lrp + rpoff[inst];
    const long long s = rp[r], e = rp[r + 1], z0 = zoff[inst];
    const int x0 = xoff[inst];
    if (lane == 0) grp[g] = z0 + s;
    for (long long k = s + lane; k < e; k += 32) {
      gci[z0 + k] = x0 + lci[z0 + k];
      rowid[z0 + k] = (int)g;
    }
  }
  if (gtid() == 0) grp[M] = Z;
}

__device__ __forceinline__ void max_into(unsigned* out, int v) {
  const int m = __reduce_max_sync(0xffffffffu, v);
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned)m);
}

__global__ void k_row_lengths(const long long* __restrict__ rp, long long M, int* __restrict__ len,
                              unsigned* __restrict__ maxlen) {
  int mx = 0;
  for (long long i = gtid(); i < M; i += gstride()) {
    const int l = (int)(rp[i + 1] - rp[i]);
    len[i] = l;
    mx = max(mx, l);
  }
  max_into(maxlen, mx);
}

__global__ void k_col_counts(const int* __restrict__ ci, long long Z, int* __restrict__ cnt) {
  for (long long k = gtid(); k < Z; k += gstride()) atomicAdd(&cnt[ci[k]], 1);
}

__global__ void k_max_int(const int* __restrict__ v, long long len, unsigned* __restrict__ out) {
  int mx = 0;
  for (long long i = gtid(); i < len; i += gstride()) mx = max(mx, v[i]);
  max_into(out, mx);
}

// sort keys of the renumbering: instance in the high bits, then
// (maxlen - length), so that an ascending stable sort orders every instance's
// rows by decreasing length and keeps the instances in place
// sec (optional, sbits wide) is a secondary key below the length: rows of
// equal length are ordered by it (stably where it ties)
__global__ void k_length_keys(const int* __restrict__ len, long long cnt, const int* __restrict__ inst, int maxlen,
                              int lbits, const int* __restrict__ sec, int sbits, unsigned long long* __restrict__ keys,
                              int* __restrict__ vals) {
  for (long long i = gtid(); i < cnt; i += gstride()) {
    const unsigned long long hi = inst ? (unsigned long long)inst[i] : 0ull;
    const unsigned long long lo = sec ? (unsigned long long)(unsigned)sec[i] : 0ull;
    keys[i] = (((hi << lbits) | (unsigned long long)(maxlen - len[i])) << sbits) | lo;
    vals[i] = (int)i;
  }
}

// secondary sort key of the columns: the internal row of a column's only
// entry for one-entry columns, 0 for the others (sec zeroed before)
__global__ void k_singleton_rows(const int* __restrict__ gci, const int* __restrict__ rowid, long long Z,
                                 const int* __restrict__ lenT, const int* __restrict__ iy, int* __restrict__ sec) {
  for (long long k = gtid(); k < Z; k += gstride()) {
    const int c = gci[k];
    if (lenT[c] == 1) sec[c] = iy[rowid[k]];
  }
}

// sort keys of the transpose, fed in internal row order (internal row r =
// the caller's row py[r], entries from grp[py[r]]; rpi: its exclusive scan of
// lengths), so that every row of A^T lists its entries by increasing
// internal row: entry k goes to the row of its internal column
__global__ void k_transpose_keys(const long long* __restrict__ grp, const int* __restrict__ py,
                                 const long long* __restrict__ rpi, long long M, const int* __restrict__ gci,
                                 const int* __restrict__ ix, unsigned* __restrict__ keys, int* __restrict__ vals) {
  const int lane = threadIdx.x & 31;
  const long long w0 = gtid() >> 5, nw = gstride() >> 5;
  for (long long r = w0; r < M; r += nw) {
    const long long s = grp[py[r]], len = rpi[r + 1] - rpi[r], o = rpi[r];
    for (long long e = lane; e < len; e += 32) {
      const long long k = s + e;
      keys[o + e] = (unsigned)ix[gci[k]];
      vals[o + e] = (int)k;
    }
  }
}

// ---- panel layout of A^T (panel-tiled primal step) ---------------------------

// panel p holds the internal rows [pfirst[p], pfirst[p + 1]); the panel of row i
__device__ __forceinline__ int panel_of(const int* __restrict__ pfirst, int P, int i) {
  int lo = 0, hi = P;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pfirst[mid] <= i)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// cnt[i] += the entries of A^T's first rows (positions [0, Z) of the sorted
// A^T entries) in internal row i of A: the weights of the panel heights
__global__ void k_row_counts(long long Z, const int* __restrict__ sval, const int* __restrict__ rowid,
                             const int* __restrict__ iy, int* __restrict__ cnt) {
  for (long long q = gtid(); q < Z; q += gstride()) atomicAdd(cnt + iy[rowid[sval[q]]], 1);
}

// head[p] = 1 where a segment (a maximal run of one row of A^T inside one
// panel) starts; panel[p] = its panel
__global__ void k_panel_heads(const long long* __restrict__ tp, long long N, const int* __restrict__ sval,
                              const int* __restrict__ rowid, const int* __restrict__ iy,
                              const int* __restrict__ pfirst, int P, int* __restrict__ head, int* __restrict__ panel,
                              int* __restrict__ col) {
  const int lane = threadIdx.x & 31;
  const long long w0 = gtid() >> 5, nw = gstride() >> 5;
  for (long long j = w0; j < N; j += nw) {
    const long long a = tp[j], b = tp[j + 1];
    for (long long q = a + lane; q < b; q += 32) {
      const int pq = panel_of(pfirst, P, iy[rowid[sval[q]]]);
      const int pp = q > a ? panel_of(pfirst, P, iy[rowid[sval[q - 1]]]) : -1;
      head[q] = pq != pp;
      panel[q] = pq;
      col[q] = (int)j;
    }
  }
}

// per segment s (numbered in order of position, i.e. column by column): its
// first position, panel and column; segpos = exclusive scan of head
__global__ void k_panel_segments(const int* __restrict__ head, const int* __restrict__ panel,
                                 const int* __restrict__ col, const long long* __restrict__ segpos, long long Z,
                                 long long S, long long* __restrict__ seg_start, int* __restrict__ seg_panel,
                                 int* __restrict__ seg_col) {
  for (long long q = gtid(); q < Z; q += gstride())
    if (head[q]) {
      const long long sid = segpos[q];
      seg_start[sid] = q;
      seg_panel[sid] = panel[q];
      seg_col[sid] = col[q];
    }
  if (gtid() == 0) seg_start[S] = Z;
}

__global__ void k_panel_keys(const long long* __restrict__ seg_start, const int* __restrict__ seg_panel, long long S,
                             int maxlen, int lbits, int* __restrict__ seg_len, unsigned long long* __restrict__ keys,
                             int* __restrict__ vals, int* __restrict__ pcount) {
  for (long long sid = gtid(); sid < S; sid += gstride()) {
    const int len = (int)(seg_start[sid + 1] - seg_start[sid]);
    seg_len[sid] = len;
    keys[sid] = ((unsigned long long)seg_panel[sid] << lbits) | (unsigned long long)(maxlen - len);
    vals[sid] = (int)sid;
    atomicAdd(&pcount[seg_panel[sid]], 1);
  }
}

// column and first row of A of every segment row r (segment sp[r])
__global__ void k_panel_rowinfo(const int* __restrict__ sp, const int* __restrict__ seg_col,
                                const int* __restrict__ seg_panel, const int* __restrict__ pfirst, long long S,
                                int* __restrict__ pcol, int* __restrict__ pbase) {
  for (long long r = gtid(); r < S; r += gstride()) {
    const int sid = sp[r];
    pcol[r] = seg_col[sid];
    pbase[r] = pfirst[seg_panel[sid]];
  }
}

// partial-sum position of every segment row r in the dense panel-major array
// of the panel pass: panel * ncols + column
__global__ void k_panel_dense_out(const int* __restrict__ pcol, const int* __restrict__ sp,
                                  const int* __restrict__ seg_panel, int ncols, long long S, int* __restrict__ out) {
  for (long long r = gtid(); r < S; r += gstride()) out[r] = seg_panel[sp[r]] * ncols + pcol[r];
}

__global__ void k_invert(const int* __restrict__ p, long long len, int* __restrict__ inv) {
  for (long long i = gtid(); i < len; i += gstride()) inv[p[i]] = (int)i;
}

template <class T>
__global__ void k_gather(const T* __restrict__ src, const int* __restrict__ p, long long len, T* __restrict__ out) {
  for (long long i = gtid(); i < len; i += gstride()) out[i] = src[p[i]];
}

// ---- stable LSD radix sort of (key, value) pairs, 8 bits per pass ------------

// per-block digit counts, stored digit-major: hist[d * nblocks + block]
template <class K>
__global__ void __launch_bounds__(RS_TPB) k_rs_hist(const K* __restrict__ keys, long long N, int shift,
                                                    long long* __restrict__ hist, int nblocks) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * RS_TILE;
  for (int it = 0; it < RS_ITEMS; ++it) {
    const long long i = base + (long long)it * RS_TPB + threadIdx.x;
    if (i < N) atomicAdd(&h[(int)((keys[i] >> shift) & 255u)], 1);
  }
  __syncthreads();
  hist[(long long)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Scatter of one pass. offs = exclusive scan of hist, so offs[d * nblocks + b]
// is where block b's first key with digit d goes. Within a block the keys are
// ranked in index order: round by round, warp by warp, lane by lane (lanes
// with the same digit found with match.any), which makes the pass stable.
template <class K>
__global__ void __launch_bounds__(RS_TPB) k_rs_scatter(const K* __restrict__ kin, const int* __restrict__ vin,
                                                       K* __restrict__ kout, int* __restrict__ vout, long long N,
                                                       int shift, const long long* __restrict__ offs, int nblocks) {
  constexpr int NW = RS_TPB / 32;
  __shared__ long long s_base[256];
  __shared__ int s_run[256];
  __shared__ int s_w[NW][256];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  s_base[t] = offs[(long long)t * nblocks + blockIdx.x];
  s_run[t] = 0;
  const unsigned below = (1u << lane) - 1u;
  const long long base = (long long)blockIdx.x * RS_TILE;
  for (int it = 0; it < RS_ITEMS; ++it) {
    __syncthreads();  // the previous round's reads of s_w are done
#pragma unroll
    for (int w = 0; w < NW; ++w) s_w[w][t] = 0;
    const long long i = base + (long long)it * RS_TPB + t;
    const bool valid = i < N;
    K key = 0;
    int val = 0, d = 256;  // 256: no key in this slot
    if (valid) {
      key = kin[i];
      val = vin[i];
      d = (int)((key >> shift) & 255u);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & below);
    __syncthreads();
    if (valid && rank == 0) s_w[warp][d] = __popc(peers);
    __syncthreads();
    {
      int acc = s_run[t];
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        const int c = s_w[w][t];
        s_w[w][t] = acc;
        acc += c;
      }
      s_run[t] = acc;
    }
    __syncthreads();
    if (valid) {
      const long long pos = s_base[d] + s_w[warp][d] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
  }
}

// ---- exclusive scan (len inputs -> len + 1 outputs, out[len] = total) --------

template <class T>
__global__ void __launch_bounds__(SC_TPB) k_scan_tile(const T* __restrict__ in, long long len,
                                                      long long* __restrict__ out, long long* __restrict__ tsum) {
  __shared__ long long wsum[SC_TPB / 32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const long long base = (long long)blockIdx.x * SC_TILE + (long long)t * SC_ITEMS;
  long long v[SC_ITEMS];
  long long sum = 0;
#pragma unroll
  for (int j = 0; j < SC_ITEMS; ++j) {
    const long long i = base + j;
    v[j] = i < len ? (long long)in[i] : 0;
    sum += v[j];
  }
  long long x = sum;  // inclusive scan within the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  long long before = 0, total = 0;
  for (int w = 0; w < SC_TPB / 32; ++w) {
    if (w < warp) before += wsum[w];
    total += wsum[w];
  }
  long long run = before + x - sum;
#pragma unroll
  for (int j = 0; j < SC_ITEMS; ++j) {
    const long long i = base + j;
    if (i <= len) out[i] = run;
    run += v[j];
  }
  if (t == 0) tsum[blockIdx.x] = total;
}

__global__ void k_scan_add(long long* __restrict__ out, long long count, const long long* __restrict__ toff) {
  for (long long i = gtid(); i < count; i += gstride()) out[i] += toff[i / SC_TILE];
}

long long scan_tiles(long long len) { return (len + 1 + SC_TILE - 1) / SC_TILE; }

template <class T>
void scan_exclusive(const T* in, long long len, long long* out, long long* ws, cudaStream_t s) {
  const long long tiles = scan_tiles(len);
  k_scan_tile<T><<<(unsigned)tiles, SC_TPB, 0, s>>>(in, len, out, ws);
  if (tiles > 1) {
    long long* toff = ws + tiles;  // tiles + 1 entries
    scan_exclusive<long long>(ws, tiles, toff, toff + tiles + 1, s);
    k_scan_add<<<grid_of(len + 1), LT_TPB, 0, s>>>(out, len + 1, toff);
  }
}

// ---- packing of the units -----------------------------------------------------

// entries of internal row `row` of A: the caller's row py[row]
struct SrcA {
  const long long* grp;
  const int* py;
  const int* gci;
  const int* ix;
  const double* v;
  __device__ long long start(int row) const { return grp[py[row]]; }
  __device__ void get(int, long long p, int& c, double& x) const {
    c = ix[gci[p]];
    x = v[p];
  }
};

// entries of internal row `row` of A^T: positions [tp[row], tp[row + 1]) of
// the entries sorted by internal column
struct SrcT {
  const long long* tp;
  const int* sval;
  const int* rowid;
  const int* iy;
  const double* v;
  __device__ long long start(int row) const { return tp[row]; }
  __device__ void get(int, long long p, int& c, double& x) const {
    const int k = sval[p];
    c = iy[rowid[k]];
    x = v[k];
  }
};

// entries of segment row `row` of the panel layout: positions from
// seg_start[sp[row]] of the A^T entries (sorted by internal column, then
// internal row), with the row index taken relative to the segment's panel
struct SrcPanel {
  const int* sp;
  const long long* seg_start;
  const int* seg_panel;
  const int* sval;
  const int* rowid;
  const int* iy;
  const double* v;
  const int* pfirst;
  __device__ long long start(int row) const { return seg_start[sp[row]]; }
  __device__ void get(int row, long long p, int& c, double& x) const {
    const int k = sval[p];
    c = iy[rowid[k]] - pfirst[seg_panel[sp[row]]];
    x = v[k];
  }
};

// one warp per unit; slots not written here keep the zeros set before
template <class Src>
__global__ void k_fill_units(const int4* __restrict__ uinfo, const long long* __restrict__ uoff, int n_units,
                             const int* __restrict__ slen, Src src, int* __restrict__ ci, double* __restrict__ v) {
  const int lane = threadIdx.x & 31;
  const long long w0 = gtid() >> 5, nw = gstride() >> 5;
  for (long long u = w0; u < n_units; u += nw) {
    const int4 info = uinfo[u];
    const long long base = uoff[u], end = uoff[u + 1];
    if (info.y == 0) {
      const long long s = src.start(info.x);
      const int len = slen[info.x];
      for (int e = lane; e < len; e += 32) {
        int c;
        double x;
        src.get(info.x, s + e, c, x);
        ci[base + e] = c;
        v[base + e] = x;
      }
    } else {
      const int R = info.y;
      const int Lp = (int)((end - base) / (32 * R));
      for (int q = 0; q < R; ++q) {
        if (32 * q + lane >= info.z) continue;
        const int row = info.x + 32 * q + lane;
        const long long s = src.start(row);
        const int len = slen[row];
        for (int e = 0; e < len; ++e) {
          int c;
          double x;
          src.get(row, s + e, c, x);
          const long long k = slice_slot(base, Lp, R, q, e, lane);
          ci[k] = c;
          v[k] = x;
        }
      }
    }
  }
}

// ---- validation of a CSR held on the device -----------------------------------

__global__ void k_validate_csr(long long m, long long n, long long nnz, const long long* __restrict__ rp,
                               const int* __restrict__ ci, const double* __restrict__ v, int* __restrict__ flags) {
  const int lane = threadIdx.x & 31;
  const long long w0 = gtid() >> 5, nw = gstride() >> 5;
  int f = 0;
  for (long long i = w0; i < m; i += nw) {
    const long long a = rp[i], b = rp[i + 1];
    bool bad = a < 0 || b > nnz || b < a;
    if (i == 0 && a != 0) bad = true;
    if (i == m - 1 && b != nnz) bad = true;
    if (bad) {
      f |= LAYOUT_BAD_ROW_PTR;
      continue;
    }
    for (long long k = a + lane; k < b; k += 32) {
      const int c = ci[k];
      if (c < 0 || c >= n) f |= LAYOUT_BAD_COLUMN;
      if (k > a && c <= ci[k - 1]) f |= LAYOUT_UNSORTED;
      if (!isfinite(v[k])) f |= LAYOUT_NOT_FINITE;
    }
  }
  f = __reduce_or_sync(0xffffffffu, f);
  if (lane == 0 && f) atomicOr(flags, f);
}

__global__ void k_check_finite(const double* __restrict__ v, long long len, int* __restrict__ flags) {
  int f = 0;
  for (long long i = gtid(); i < len; i += gstride())
    if (!isfinite(v[i])) f = LAYOUT_NOT_FINITE;
  f = __reduce_or_sync(0xffffffffu, f);
  if ((threadIdx.x & 31) == 0 && f) atomicOr(flags, f);
}

}  // namespace

// ---- launchers ------------------------------------------------------------------

void launch_instance_of(const int* off, int count, long long len, int* out, cudaStream_t s) {
  if (len > 0) k_instance_of<<<grid_of(len), LT_TPB, 0, s>>>(off, count, len, out);
}

void launch_globalize(const long long* lrp, const int* lci, const long long* rpoff, const long long* zoff,
                      const int* xoff, const int* yoff, const int* rinst, long long M, long long Z, long long* grp,
                      int* gci, int* rowid, cudaStream_t s) {
  k_globalize<<<grid_of(32 * M), LT_TPB, 0, s>>>(lrp, lci, rpoff, zoff, xoff, yoff, rinst, M, Z, grp, gci, rowid);
}

void launch_lengths(const long long* grp, long long M, const int* gci, long long Z, long long N, int* lenA,
                    int* lenT, unsigned* maxes, cudaStream_t s) {
  cudaMemsetAsync(maxes, 0, 2 * sizeof(unsigned), s);
  cudaMemsetAsync(lenT, 0, sizeof(int) * N, s);
  k_row_lengths<<<grid_of(M), LT_TPB, 0, s>>>(grp, M, lenA, maxes);
  if (Z > 0) k_col_counts<<<grid_of(Z), LT_TPB, 0, s>>>(gci, Z, lenT);
  k_max_int<<<grid_of(N), LT_TPB, 0, s>>>(lenT, N, maxes + 1);
}

void launch_length_keys(const int* len, long long cnt, const int* inst, int maxlen, int lbits,
                        unsigned long long* keys, int* vals, cudaStream_t s, const int* sec, int sbits) {
  k_length_keys<<<grid_of(cnt), LT_TPB, 0, s>>>(len, cnt, inst, maxlen, lbits, sec, sbits, keys, vals);
}

void launch_singleton_rows(const int* gci, const int* rowid, long long Z, const int* lenT, const int* iy, int* sec,
                           long long N, cudaStream_t s) {
  cudaMemsetAsync(sec, 0, sizeof(int) * N, s);
  if (Z > 0) k_singleton_rows<<<grid_of(Z), LT_TPB, 0, s>>>(gci, rowid, Z, lenT, iy, sec);
}

void launch_transpose_keys(const long long* grp, const int* py, const long long* rpi, long long M, const int* gci,
                           const int* ix, unsigned* keys, int* vals, cudaStream_t s) {
  k_transpose_keys<<<grid_of(32 * M), LT_TPB, 0, s>>>(grp, py, rpi, M, gci, ix, keys, vals);
}

void launch_row_counts(long long Z, const int* sval, const int* rowid, const int* iy, int* cnt, cudaStream_t s) {
  if (Z > 0) k_row_counts<<<grid_of(Z), LT_TPB, 0, s>>>(Z, sval, rowid, iy, cnt);
}

void launch_panel_heads(const long long* tp, long long N, const int* sval, const int* rowid, const int* iy,
                        const int* pfirst, int P, int* head, int* panel, int* col, cudaStream_t s) {
  k_panel_heads<<<grid_of(32 * N), LT_TPB, 0, s>>>(tp, N, sval, rowid, iy, pfirst, P, head, panel, col);
}

void launch_panel_segments(const int* head, const int* panel, const int* col, const long long* segpos, long long Z,
                           long long S, long long* seg_start, int* seg_panel, int* seg_col, cudaStream_t s) {
  k_panel_segments<<<grid_of(std::max(1LL, Z)), LT_TPB, 0, s>>>(head, panel, col, segpos, Z, S, seg_start, seg_panel,
                                                                 seg_col);
}

void launch_panel_rowinfo(const int* sp, const int* seg_col, const int* seg_panel, const int* pfirst, long long S,
                          int* pcol, int* pbase, cudaStream_t s) {
  if (S > 0) k_panel_rowinfo<<<grid_of(S), LT_TPB, 0, s>>>(sp, seg_col, seg_panel, pfirst, S, pcol, pbase);
}

void launch_panel_keys(const long long* seg_start, const int* seg_panel, long long S, int maxlen, int lbits,
                       int* seg_len, unsigned long long* keys, int* vals, int* pcount, cudaStream_t s) {
  if (S > 0) k_panel_keys<<<grid_of(S), LT_TPB, 0, s>>>(seg_start, seg_panel, S, maxlen, lbits, seg_len, keys, vals,
                                                         pcount);
}

void launch_panel_dense_out(const int* pcol, const int* sp, const int* seg_panel, int ncols, long long S, int* out,
                            cudaStream_t s) {
  if (S > 0) k_panel_dense_out<<<grid_of(S), LT_TPB, 0, s>>>(pcol, sp, seg_panel, ncols, S, out);
}

void launch_max_int(const int* v, long long len, unsigned* out, cudaStream_t s) {
  cudaMemsetAsync(out, 0, sizeof(unsigned), s);
  if (len > 0) k_max_int<<<grid_of(len), LT_TPB, 0, s>>>(v, len, out);
}

void launch_fill_units_P(const Hyb& H, const int* slen, const int* sp, const long long* seg_start,
                         const int* seg_panel, const int* sval, const int* rowid, const int* iy, const double* v,
                         const int* pfirst, cudaStream_t s) {
  if (H.n_units == 0) return;
  SrcPanel src{sp, seg_start, seg_panel, sval, rowid, iy, v, pfirst};
  k_fill_units<SrcPanel><<<grid_of(32LL * H.n_units), LT_TPB, 0, s>>>(H.uinfo, H.uoff, H.n_units, slen, src, H.ci,
                                                                      H.v);
}

void launch_invert(const int* p, long long len, int* inv, cudaStream_t s) {
  k_invert<<<grid_of(len), LT_TPB, 0, s>>>(p, len, inv);
}

void launch_gather_int(const int* src, const int* p, long long len, int* out, cudaStream_t s) {
  if (len > 0) k_gather<int><<<grid_of(len), LT_TPB, 0, s>>>(src, p, len, out);
}

void launch_gather_double(const double* src, const int* p, long long len, double* out, cudaStream_t s) {
  if (len > 0) k_gather<double><<<grid_of(len), LT_TPB, 0, s>>>(src, p, len, out);
}

long long radix_hist_len(long long N) { return 256LL * std::max(1LL, (N + RS_TILE - 1) / RS_TILE) + 1; }

long long scan_ws_len(long long len) {
  long long total = 0;
  for (long long l = len;;) {
    const long long t = scan_tiles(l);
    total += t + (t > 1 ? t + 1 : 0);
    if (t <= 1) break;
    l = t;
  }
  return total + 8;
}

template <class K>
int radix_sort_pairs(K* keys, int* vals, K* keys_alt, int* vals_alt, long long N, int bits, long long* hist,
                     long long* ws, cudaStream_t s) {
  const int nblocks = (int)std::max(1LL, (N + RS_TILE - 1) / RS_TILE);
  int passes = 0;
  K* ka = keys;
  int* va = vals;
  K* kb = keys_alt;
  int* vb = vals_alt;
  for (int shift = 0; shift < bits && N > 1; shift += 8, ++passes) {
    k_rs_hist<K><<<nblocks, RS_TPB, 0, s>>>(ka, N, shift, hist, nblocks);
    scan_exclusive<long long>(hist, 256LL * nblocks, hist, ws, s);
    k_rs_scatter<K><<<nblocks, RS_TPB, 0, s>>>(ka, va, kb, vb, N, shift, hist, nblocks);
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  return passes & 1;
}

template int radix_sort_pairs<unsigned>(unsigned*, int*, unsigned*, int*, long long, int, long long*, long long*,
                                        cudaStream_t);
template int radix_sort_pairs<unsigned long long>(unsigned long long*, int*, unsigned long long*, int*, long long,
                                                  int, long long*, long long*, cudaStream_t);

void launch_scan_int(const int* in, long long len, long long* out, long long* ws, cudaStream_t s) {
  scan_exclusive<int>(in, len, out, ws, s);
}

void launch_fill_units_A(const Hyb& H, const int* slen, const long long* grp, const int* py, const int* gci,
                         const int* ix, const double* v, cudaStream_t s) {
  if (H.n_units == 0) return;
  SrcA src{grp, py, gci, ix, v};
  k_fill_units<SrcA><<<grid_of(32LL * H.n_units), LT_TPB, 0, s>>>(H.uinfo, H.uoff, H.n_units, slen, src, H.ci, H.v);
}

void launch_fill_units_T(const Hyb& H, const int* slen, const long long* tp, const int* sval, const int* rowid,
                         const int* iy, const double* v, cudaStream_t s) {
  if (H.n_units == 0) return;
  SrcT src{tp, sval, rowid, iy, v};
  k_fill_units<SrcT><<<grid_of(32LL * H.n_units), LT_TPB, 0, s>>>(H.uinfo, H.uoff, H.n_units, slen, src, H.ci, H.v);
}

void launch_validate_csr(long long m, long long n, long long nnz, const long long* rp, const int* ci,
                         const double* v, int* flags, cudaStream_t s) {
  k_validate_csr<<<grid_of(32 * m), LT_TPB, 0, s>>>(m, n, nnz, rp, ci, v, flags);
}

void launch_check_finite(const double* v, long long len, int* flags, cudaStream_t s) {
  if (len > 0) k_check_finite<<<grid_of(len), LT_TPB, 0, s>>>(v, len, flags);
}

}  // namespace pdhg
