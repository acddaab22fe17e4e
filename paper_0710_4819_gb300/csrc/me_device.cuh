// me_device.cuh -- device building blocks of the block-matching kernels:
// the packed-byte SAD step, the rate term, the packed argmin key and the
// CTA-wide full search of one block.  Included by the .cu files of the
// library only (not part of the C ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace me {

constexpr int kMaxP = 64;
constexpr int kMaxThreads = 512;
constexpr unsigned long long kNoKey = ~0ull;

// One packed-byte SAD step: c + sum_k |a.byte[k] - b.byte[k]|  (eq. SAD, Sec. 2.1,
// four pixels at a time).  One instruction of the integer pipe at 16 lanes per
// clock per SM sub-partition on sm_103a.
__device__ __forceinline__ uint32_t sad4(uint32_t a, uint32_t b, uint32_t c) {
  // the accumulator is one read-write operand, so it can stay in one register
  asm("vabsdiff4.u32.u32.u32.add %0, %1, %2, %0;" : "+r"(c) : "r"(a), "r"(b));
  return c;
}

// The first step of an accumulation (accumulator zero): the zero can be the
// zero register, so no register has to be cleared per candidate.
__device__ __forceinline__ uint32_t sad4_first(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("vabsdiff4.u32.u32.u32.add %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(0u));
  return d;
}

// Bits of the signed Exp-Golomb code of one MV component: 1 for 0, else
// 2*floor(log2|v|) + 3.  R(mv) of eq. J is mv_bits(mvx) + mv_bits(mvy).
__host__ __device__ __forceinline__ int mv_bits(int v) {
  unsigned a = v < 0 ? (unsigned)(-v) : (unsigned)v;
  if (a == 0) return 1;
#ifdef __CUDA_ARCH__
  return 2 * (31 - __clz((int)a)) + 3;
#else
  int lg = 0;
  while (a > 1u) { a >>= 1; lg++; }
  return 2 * lg + 3;
#endif
}

// The total order on candidates as one 64-bit key (smaller wins):
// J_q8 in the high word; then |mvx|+|mvy|; then the raster index of the
// position in the (2p+1)^2 window, (mvy+p)*(2p+1) + (mvx+p), which orders by
// mvy, then mvx.  J_q8 < 2^26, |mv|_1 <= 128, raster < 2^15.
__host__ __device__ __forceinline__ unsigned long long make_key(uint32_t J, int mvx, int mvy, int p) {
  uint32_t l1 = (uint32_t)((mvx < 0 ? -mvx : mvx) + (mvy < 0 ? -mvy : mvy));
  uint32_t r = (uint32_t)((mvy + p) * (2 * p + 1) + (mvx + p));
  return ((unsigned long long)J << 32) | ((unsigned long long)l1 << 17) | r;
}

struct Decoded {
  int mvx, mvy;
  uint32_t J, sad;
};

// Inverse of make_key; SAD follows exactly from J = 256*SAD + lambda*R.
__host__ __device__ __forceinline__ Decoded decode_key(unsigned long long key, int p, uint32_t lam) {
  Decoded d;
  uint32_t r = (uint32_t)(key & 0x1FFFFu);
  int n = 2 * p + 1;
  d.mvy = (int)(r / (uint32_t)n) - p;
  d.mvx = (int)(r % (uint32_t)n) - p;
  d.J = (uint32_t)(key >> 32);
  d.sad = (d.J - lam * (uint32_t)(mv_bits(d.mvx) + mv_bits(d.mvy))) >> 8;
  return d;
}

__device__ __forceinline__ unsigned long long umin64(unsigned long long a, unsigned long long b) {
  return a < b ? a : b;
}

__device__ __forceinline__ unsigned long long warp_min64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = umin64(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// The same minimum in two 32-bit warp reductions (high word, then the low
// word among the lanes holding the least high word).  Every lane of the warp
// must call it.
__device__ __forceinline__ unsigned long long warp_min64_redux(unsigned long long v) {
  const unsigned hi = (unsigned)(v >> 32);
  const unsigned mhi = __reduce_min_sync(0xffffffffu, hi);
  const unsigned lo = hi == mhi ? (unsigned)v : 0xffffffffu;
  const unsigned mlo = __reduce_min_sync(0xffffffffu, lo);
  return ((unsigned long long)mhi << 32) | mlo;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// ---------------------------------------------------------------------------
// Full search (Sec. 2.3) of a group of horizontally adjacent blocks by one CTA.
//
// The CTA stages the union of the blocks' search windows once (rows clamped to
// the frame; columns read as aligned 32-bit words, clamped byte by byte only
// when the window crosses the left or right frame edge), then re-lays it out
// as "shifted words": sh[r][o] holds window bytes o..o+3 of row r, so a
// candidate at any horizontal offset reads its reference row as N/4 aligned
// words with no byte shuffling, and consecutive offsets hit consecutive banks.
//
// Work split: G threads per block (G = 8, 16, 32, or a multiple of 32), so the
// CTA holds bpc = blockDim/G blocks.  A task is (mvx column, run of T
// consecutive mvy) of one block.  A thread keeps its N x M current block in
// registers (loaded once) and streams the T+M-1 reference rows of each run:
// reference row r serves every candidate k of the run with j = r - k in [0, M),
// so each reference word is loaded once per run and reused by up to min(T, M)
// candidates.  Tasks are dealt round-robin to the G threads of the block
// (consecutive threads take consecutive columns).
// ---------------------------------------------------------------------------
struct FsGeom {
  int p, n;          // search range, n = 2p+1 positions per axis
  int c0, nc;        // the mvx columns searched: c0 .. c0+nc-1 (mvx = column - p)
  int rb;            // bits of the per-run tie rank (0: use 64-bit keys throughout)
  int nseg;          // runs per column: ceil(n / T)
  int bpc;           // blocks in this group (adjacent, same block row)
  int G;             // threads per block
  int rows;          // staged window rows: nseg*T + M - 1
  int pos;           // shifted-word positions per row
  int sp;            // shifted-word row pitch in words (>= pos)
  int wbw;           // 32-bit words per staged raw row
  int wbp;           // the same when staged from a padded reference (16-byte chunks)
  int tasks;         // tasks per block: n * nseg
};

// Bits of the rank 2|mvy| - [mvy < 0] (0 .. 2p) that orders equal costs
// within a run (fixed mvx): smaller |mvy| first, then the negative one.
__host__ __device__ inline int rank_bits(int p) {
  int b = 0;
  while ((1 << b) <= 2 * p) b++;
  return b;
}

// Whether (J_q8 << rank_bits) + rank fits in 32 bits for every candidate, so a
// run can be reduced with 32-bit minima: J_q8 <= 256*255*N*M + lambda*R_max.
__host__ __device__ inline bool fast32_ok(int N, int M, int p, uint32_t lam) {
  const unsigned long long jmax =
      256ull * 255ull * (unsigned long long)(N * M) + (unsigned long long)lam * (2ull * mv_bits(p));
  const int rb = rank_bits(p);
  return ((jmax << rb) | ((1ull << rb) - 1)) < (1ull << 32);
}

// Bits that hold |mvy| <= p.
__host__ __device__ inline int abs_bits(int p) {
  int b = 0;
  while ((1 << b) <= p) b++;
  return b;
}

// How the runs are reduced to their best key:
//   1: 32-bit minima of (J_q8 << rank_bits) + rank for every run (fast32_ok);
//   2: 32-bit minima of (J_q8 << abs_bits) + |mvy| for the runs whose
//      candidates lie on one side of mvy = 0 (within such a run the tie
//      order is by |mvy| alone), 64-bit keys for the one run per column that
//      holds both signs -- when the |mvy| form fits 32 bits (large p);
//   0: 64-bit keys for every run.
__host__ __device__ inline int key_mode(int N, int M, int p, uint32_t lam) {
  if (fast32_ok(N, M, p, lam)) return 1;
  const unsigned long long jmax =
      256ull * 255ull * (unsigned long long)(N * M) + (unsigned long long)lam * (2ull * mv_bits(p));
  const int ab = abs_bits(p);
  return ((jmax << ab) | ((1ull << ab) - 1)) < (1ull << 32) ? 2 : 0;
}

// Per-row entry of the 32-bit run key table for key mode `mode` (tabJ =
// lambda * L(mvy) of the row).
__host__ __device__ inline uint32_t tabq_value(int mode, uint32_t tabJ, int mvy, int p) {
  const int a = mvy < 0 ? -mvy : mvy;
  if (mode == 2) return (tabJ << abs_bits(p)) + (uint32_t)a;
  return (tabJ << rank_bits(p)) + (uint32_t)(2 * a - (mvy < 0 ? 1 : 0));
}

// Geometry of a search over columns c0 .. c0+nc-1 of the (2p+1)-wide window
// (nc = 0: all columns); a slice lets several CTAs share one block's search.
// sp_min > 0 widens the shifted-word rows to a fixed pitch (a kernel compiled
// for that pitch addresses every row with immediate offsets).
template <int N, int M, int T>
__host__ __device__ inline FsGeom fs_geom(int p, int bpc, int G, int c0 = 0, int nc = 0,
                                          int sp_min = 0) {
  FsGeom g;
  g.p = p;
  g.rb = 0;
  g.n = 2 * p + 1;
  g.c0 = c0;
  g.nc = nc > 0 ? nc : g.n;
  g.nseg = (g.n + T - 1) / T;
  g.bpc = bpc;
  g.G = G;
  g.rows = g.nseg * T + M - 1;
  // position o = blk*N + col (col < nc) is read as words o .. o+N-4
  g.pos = (bpc - 1) * N + g.nc + N - 4;
  // raw row: up to 3 bytes of alignment slack, pos+3 bytes, one spare word
  g.wbw = (g.pos + 6) / 4 + 1;
  // padded staging: up to 15 bytes of alignment slack, pos+3 bytes, one spare word
  g.wbp = 4 * ((15 + g.pos + 3 + 4 + 15) / 16);
  g.sp = g.pos > sp_min ? g.pos : sp_min;
  g.tasks = g.nc * g.nseg;
  return g;
}

// Shared-memory bytes used by fs_group for a geometry.
template <int N, int M, int T>
__host__ __device__ inline size_t fs_smem_bytes(const FsGeom& g) {
  size_t words = (size_t)g.bpc * M * (N / 4)        // current blocks
               + (size_t)g.rows * (g.wbw > g.wbp ? g.wbw : g.wbp)   // raw window
               + (size_t)g.rows * g.sp              // shifted words
               + (size_t)g.rows * 3;                // per-row rate/key tables
  return words * 4 + 16 * 8 + 8;                    // per-block minima (+ alignment)
}

// The SADs of one run: T candidates of one mvx column, consecutive mvy,
// against the shifted-word rows at shp (pitch sp words).  c holds the
// block's current pixels as packed words.  Reference row r serves every
// candidate k with j = r - k in [0, M); word-major order puts consecutive SAD
// steps on different candidates.
template <int N, int M, int T>
__device__ __forceinline__ void fs_run_sads(const uint32_t (&c)[M][N / 4], const uint32_t* shp,
                                            int sp, uint32_t (&acc)[T]) {
  constexpr int NW = N / 4;
#pragma unroll
  for (int r = 0; r < T + M - 1; r++) {
    uint32_t rw[NW];
#pragma unroll
    for (int w = 0; w < NW; w++) rw[w] = shp[r * sp + 4 * w];
#pragma unroll
    for (int w = 0; w < NW; w++) {
#pragma unroll
      for (int k = 0; k < T; k++) {
        const int j = r - k;
        if (j == 0 && w == 0)
          acc[k] = sad4_first(c[0][0], rw[0]);
        else if (j >= 0 && j < M)
          acc[k] = sad4(c[j][w], rw[w], acc[k]);
      }
    }
  }
}

// A shared-memory word read that the compiler keeps in program order (a
// volatile load): fs_run_sads_lr issues each row's words where the row is
// first needed, so that at most T + 1 reference rows are live in registers.
__device__ __forceinline__ uint32_t lds_ordered(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.volatile.shared.u32 %0, [%1];"
               : "=r"(v)
               : "r"((unsigned)__cvta_generic_to_shared(p)));
  return v;
}

// The same SADs with the current block read from shared memory (cs: [M][N/4]
// packed words) one row at a time instead of held in registers: current row
// j meets reference rows j .. j+T-1, so only those (and the next row, loaded
// one step ahead) stay in registers, and each enters once.  About N*M/4
// fewer registers than fs_run_sads at the same loads per run, for kernels
// that keep more warps resident.  Same sums (integer additions in another
// order).
template <int N, int M, int T>
__device__ __forceinline__ void fs_run_sads_lr(const uint32_t* cs, const uint32_t* shp, int sp,
                                               uint32_t (&acc)[T]) {
  constexpr int NW = N / 4;
  uint32_t rr[T + M][NW];
#pragma unroll
  for (int r = 0; r < T; r++)
#pragma unroll
    for (int w = 0; w < NW; w++) rr[r][w] = lds_ordered(shp + r * sp + 4 * w);
#pragma unroll
  for (int j = 0; j < M; j++) {
    if (j + T < T + M - 1) {
#pragma unroll
      for (int w = 0; w < NW; w++) rr[j + T][w] = lds_ordered(shp + (j + T) * sp + 4 * w);
    }
    uint32_t cw[NW];
#pragma unroll
    for (int w = 0; w < NW; w++) cw[w] = lds_ordered(cs + j * NW + w);
#pragma unroll
    for (int w = 0; w < NW; w++) {
#pragma unroll
      for (int k = 0; k < T; k++) {
        if (j == 0 && w == 0)
          acc[k] = sad4_first(cw[0], rr[k][0]);
        else
          acc[k] = sad4(cw[w], rr[j + k][w], acc[k]);
      }
    }
  }
}

// The best key of one run (candidates row0 .. row0+T-1 of window column wcol,
// those past row n-1 skipped), reduced as key mode `mode` says (key_mode):
// 32-bit minima using tabQ where the mode allows it for this run, else
// 64-bit keys from tabJ / tabK.
template <int T>
__device__ __forceinline__ unsigned long long fs_run_key(const uint32_t (&acc)[T], int row0, int wcol,
                                                         int p, int n, uint32_t lam, int rb, int mode,
                                                         const uint32_t* tabJ, const uint32_t* tabK,
                                                         const uint32_t* tabQ) {
  const int mvx = wcol - p;
  const uint32_t amx = (uint32_t)(mvx < 0 ? -mvx : mvx);
  const uint32_t jx = lam * (uint32_t)mv_bits(mvx);
  unsigned long long best = kNoKey;
  // mode 2 applies to runs on one side of mvy = 0
  const bool one_side = row0 >= p || row0 + T - 1 <= p;
  if (mode == 1 || (mode == 2 && one_side)) {
    // 32-bit run minimum of (J << sb) + tie bits; the mvx part of J is the
    // same for the whole run and is added after the minimum
    const int sb = mode == 1 ? rb : 32 - __clz(p);
    uint32_t m = 0xffffffffu;
    if (row0 + T <= n) {
      // a whole run inside the window: no per-candidate bounds, and a tree
      // of three-input minima
      uint32_t v[T];
#pragma unroll
      for (int k = 0; k < T; k++) v[k] = acc[k] * (256u << sb) + tabQ[row0 + k];
      m = v[0];
#pragma unroll
      for (int k = 1; k + 1 < T; k += 2) m = __vimin3_u32(m, v[k], v[k + 1]);
      if ((T & 1) == 0) m = min(m, v[T - 1]);
    } else {
#pragma unroll
      for (int k = 0; k < T; k++) {
        const int r = row0 + k;
        if (r < n) m = min(m, acc[k] * (256u << sb) + tabQ[r]);
      }
    }
    m += jx << sb;
    const uint32_t J = m >> sb, rk = m & ((1u << sb) - 1u);
    int mvy;
    if (mode == 1)
      mvy = (rk & 1u) ? -(int)((rk + 1u) >> 1) : (int)(rk >> 1);
    else
      mvy = row0 >= p ? (int)rk : -(int)rk;
    const uint32_t lo = ((amx + (uint32_t)(mvy < 0 ? -mvy : mvy)) << 17) +
                        (uint32_t)(mvy + p) * (uint32_t)n + (uint32_t)wcol;
    best = ((unsigned long long)J << 32) | lo;
  } else {
    const uint32_t kx = (amx << 17) + (uint32_t)wcol;
#pragma unroll
    for (int k = 0; k < T; k++) {
      const int r = row0 + k;
      if (r < n) {
        const uint32_t J = acc[k] * 256u + jx + tabJ[r];
        best = umin64(best, ((unsigned long long)J << 32) | (kx + tabK[r]));
      }
    }
  }
  return best;
}

// An edge-padded copy of the reference (margin P on every side, rows of
// `pitch` bytes, 16-byte aligned; `rows` rows): when given, fs_group stages
// its window from it with asynchronous 16-byte copies (one round trip, no
// clamping) instead of from the frame.
struct FsPad {
  const uint8_t* base;
  int pitch, P, rows;
};

// Full search of g.bpc adjacent blocks whose first block has top-left pixel
// (x0, y0).  The per-block winning keys go to keys_out[0..bpc) (shared
// memory, visible to all threads on return).  Every thread of the CTA calls
// it; threads beyond bpc*G only help with staging.  SP > 0: the geometry's
// shifted-word pitch is SP (fixed at compile time), else g.sp.  STATS: also
// the sum and the minimum of the SAD over the searched positions of every
// block, to stats[2*blk] and stats[2*blk+1] (shared memory, 2*bpc words).
// VOL: instead of keys, every candidate's SAD is stored to
// vol[blk*vstride + (mvy+p)*n + (mvx+p)] (global memory, uint16: a SAD is at
// most 255*N*M = 65280); keys_out then holds no result.
template <int N, int M, int T, int SP = 0, bool STATS = false, bool VOL = false>
__device__ void fs_group(const uint8_t* __restrict__ cur, const uint8_t* __restrict__ ref,
                         int W, int H, int x0, int y0, const FsGeom& g, uint32_t lam,
                         uint32_t* smem, unsigned long long* keys_out,
                         unsigned long long* tr = nullptr, FsPad pad = FsPad{nullptr, 0, 0, 0},
                         uint32_t* stats = nullptr, uint16_t* __restrict__ vol = nullptr,
                         int vstride = 0) {
  constexpr int NW = N / 4;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nthr >> 5;
  const int p = g.p, n = g.n;
  const int sp = SP > 0 ? SP : g.sp;
  const int wpitch = pad.base ? g.wbp : g.wbw;             // staged raw row pitch (words)
  uint32_t* curw = smem;                                   // [bpc][M][NW]
  uint32_t* wb = curw + g.bpc * M * NW;                    // [rows][wpitch]
  uint32_t* sh = wb + g.rows * (g.wbw > g.wbp ? g.wbw : g.wbp);   // [rows][sp]
  uint32_t* tabJ = sh + g.rows * sp;                    // [rows] lambda*L(mvy)
  uint32_t* tabK = tabJ + g.rows;                          // [rows] key bits of mvy
  uint32_t* tabQ = tabK + g.rows;                          // [rows] 32-bit run key of mvy
  unsigned long long* red = reinterpret_cast<unsigned long long*>(
      (reinterpret_cast<uintptr_t>(tabQ + g.rows) + 7) & ~uintptr_t(7));
  const int fast = key_mode(N, M, p, lam);
  const int rb = rank_bits(p);

  if (tid < g.bpc) red[tid] = kNoKey;
  if (STATS && tid < g.bpc) {
    stats[2 * tid] = 0u;
    stats[2 * tid + 1] = 0xffffffffu;
  }
  int s0;
  if (pad.base) {
    // 1+2 from the padded reference: current blocks as 4-byte and window rows
    // as 16-byte asynchronous copies, all in flight together
    for (int i = tid; i < g.bpc * M * NW; i += nthr) {
      const int blk = i / (M * NW), rem = i % (M * NW), j = rem / NW, w = rem % NW;
      const unsigned dst = (unsigned)__cvta_generic_to_shared(curw + i);
      const void* src = cur + (size_t)(y0 + j) * W + x0 + blk * N + 4 * w;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
    }
    const int X = x0 + pad.P - p + g.c0;  // padded column of window column 0
    const int A = X & ~15;
    s0 = X - A;
    const int cw = g.wbp / 4;              // 16-byte chunks per row
    for (int i = tid; i < g.rows * cw; i += nthr) {
      const int r = i / cw, c = i - r * cw;
      const int yr = min(y0 + pad.P - p + r, pad.rows - 1);   // rows past the margin: edge rows
      const unsigned dst = (unsigned)__cvta_generic_to_shared(wb + r * wpitch + 4 * c);
      const void* src = pad.base + (size_t)yr * pad.pitch + A + 16 * c;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  } else {
    // 1. current blocks (rows 4-byte aligned: W % 4 == 0, x0 % 4 == 0)
    for (int i = tid; i < g.bpc * M * NW; i += nthr) {
      const int blk = i / (M * NW), rem = i % (M * NW), j = rem / NW, w = rem % NW;
      curw[i] = *reinterpret_cast<const uint32_t*>(cur + (size_t)(y0 + j) * W + x0 + blk * N + 4 * w);
    }
    // 2. raw window rows, from the aligned word at or left of column x0 - p
    const int wx0 = x0 - p + g.c0;
    const int A0 = (wx0 >> 2) << 2;        // floor to a multiple of 4
    s0 = wx0 - A0;
    const bool inside = A0 >= 0 && A0 + 4 * g.wbw <= W;
    {
      // eight independent loads per thread in flight before their stores, so
      // the window costs about one global-memory round trip, not one per row
      const int total = g.rows * g.wbw;
      for (int base = tid; base < total; base += 8 * nthr) {
        uint32_t v[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
          const int i = base + u * nthr;
          v[u] = 0;
          if (i < total) {
            const int r = i / g.wbw, q = i - r * g.wbw;
            const uint8_t* rowp = ref + (size_t)clampi(y0 - p + r, 0, H - 1) * W;
            if (inside) {
              v[u] = *reinterpret_cast<const uint32_t*>(rowp + A0 + 4 * q);
            } else {
#pragma unroll
              for (int b = 0; b < 4; b++)
                v[u] |= (uint32_t)rowp[clampi(A0 + 4 * q + b, 0, W - 1)] << (8 * b);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 8; u++) {
          const int i = base + u * nthr;
          if (i < total) wb[i] = v[u];
        }
      }
    }
  }
  // rate / key tables per staged row r (mvy = r - p; rows past 2p are padding)
  for (int r = tid; r < g.rows; r += nthr) {
    const int mvy = r - p;
    const int a = mvy < 0 ? -mvy : mvy;
    tabJ[r] = lam * (uint32_t)mv_bits(mvy);
    tabK[r] = ((uint32_t)a << 17) + (uint32_t)r * (uint32_t)n;
    tabQ[r] = tabq_value(fast, tabJ[r], mvy, p);
  }
  if (pad.base) asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  // 3. shifted words: sh[r][o] = raw bytes s0+o .. s0+o+3
  for (int r = warp; r < g.rows; r += nwarps) {
    const uint32_t* row = wb + r * wpitch;
    uint32_t* dst = sh + r * sp;
    for (int o = lane; o < g.pos; o += 32) {
      const int k = s0 + o;
      dst[o] = __funnelshift_r(row[k >> 2], row[(k >> 2) + 1], 8 * (k & 3));
    }
  }
  __syncthreads();
  // optional timeline (thread 0, global timer): window staged, runs done
  if (tr && threadIdx.x == 0) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    tr[0] = t;
  }

  // 4. tasks of this thread's block
  const int blk = tid / g.G, l = tid - blk * g.G;
  unsigned long long best = kNoKey;
  uint32_t ssum = 0u, smin = 0xffffffffu;
  if (blk < g.bpc) {
    uint32_t c[M][NW];
#pragma unroll
    for (int j = 0; j < M; j++)
#pragma unroll
      for (int w = 0; w < NW; w++) c[j][w] = curw[(blk * M + j) * NW + w];
    const int nc = g.nc;
    int seg = l / nc, col = l - (l / nc) * nc;
    const int dseg = g.G / nc, dcol = g.G - (g.G / nc) * nc;
    for (int t = l; t < g.tasks; t += g.G) {
      const int row0 = seg * T;
      const uint32_t* shp = sh + row0 * sp + blk * N + col;
      uint32_t acc[T];
      fs_run_sads<N, M, T>(c, shp, sp, acc);
      if (STATS) {
#pragma unroll
        for (int k = 0; k < T; k++)
          if (row0 + k < n) {
            ssum += acc[k];
            smin = min(smin, acc[k]);
          }
      }
      // cost and key of each candidate of the run (mvx = c0 + col - p)
      const int wcol = g.c0 + col;
      if (VOL) {
        uint16_t* vb = vol + (size_t)blk * vstride + wcol;
#pragma unroll
        for (int k = 0; k < T; k++) {
          const int r = row0 + k;
          if (r < n) vb[r * n] = (uint16_t)acc[k];
        }
      } else {
        best = umin64(best, fs_run_key<T>(acc, row0, wcol, p, n, lam, rb, fast, tabJ, tabK, tabQ));
      }
      seg += dseg;
      col += dcol;
      if (col >= nc) { col -= nc; seg++; }
    }
  }
  if (tr && threadIdx.x == 0) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    tr[1] = t;
  }
  // 5. per-block minimum (and SAD sum / minimum)
  if (g.G <= 32) {
    for (int o = g.G >> 1; o > 0; o >>= 1) {
      best = umin64(best, __shfl_xor_sync(0xffffffffu, best, o));
      if (STATS) {
        ssum += __shfl_xor_sync(0xffffffffu, ssum, o);
        smin = min(smin, __shfl_xor_sync(0xffffffffu, smin, o));
      }
    }
    if (blk < g.bpc && l == 0) {
      red[blk] = best;
      if (STATS) {
        stats[2 * blk] = ssum;
        stats[2 * blk + 1] = smin;
      }
    }
  } else {
    best = warp_min64(best);
    if (STATS) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ssum += __shfl_xor_sync(0xffffffffu, ssum, o);
        smin = min(smin, __shfl_xor_sync(0xffffffffu, smin, o));
      }
    }
    if (lane == 0 && blk < g.bpc && best != kNoKey) atomicMin(&red[blk], best);
    if (STATS && lane == 0 && blk < g.bpc) {
      atomicAdd(&stats[2 * blk], ssum);
      atomicMin(&stats[2 * blk + 1], smin);
    }
  }
  __syncthreads();
  if (tid < g.bpc) keys_out[tid] = red[tid];
  __syncthreads();
}

}  // namespace me
