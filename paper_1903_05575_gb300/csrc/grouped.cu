// Grouped quaternion GEMM: many independent problems in one persistent
// launch (the batching of the task; the paper tunes its cache blocking per
// machine, Sec. 3.2 and Sec. 5, and this is the GPU analogue: tile shapes
// chosen per size bucket from a table an autotuner fills).
//
// qgemm_grouped_prepare() validates every problem, picks its tile shape from
// the bucket table, encodes its TMA descriptors, and writes into the caller's
// workspace:
//   [counter | problem descriptors | tile list]
// The tile list holds (problem, row tile, column tile, shape) sorted by
// decreasing k, so the persistent CTAs, which take tiles from an atomic
// counter, finish the longest tiles first.  qgemm_grouped_launch() resets
// the counter and launches; both calls go on the caller's stream, so the
// launch alone can be captured in a CUDA graph and replayed.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "fp64_tile.cuh"
#include "split_core.cuh"

namespace qg {

// Digit-sliced FP64 batches (fp64_sliced.cu).
size_t sliced_grouped_workspace_bytes(const std::vector<GemmDesc> &ds);
int prepare_sliced_grouped(const std::vector<GemmDesc> &ds, int layout, unsigned char *ws,
                           size_t ws_bytes, cudaStream_t s, qgemm_grouped_plan *plan);
int launch_sliced_grouped(const qgemm_grouped_plan *plan, cudaStream_t s);


__device__ int g_grouped_error;

fp64::Operands fp64_operands(const GemmDesc &d);
bool encode_split_planes(CUtensorMap *map, const void *base, int64_t kq, int64_t kp,
                         int64_t rows, int planes, int box_rows);
bool encode_fp64_operand(CUtensorMap *map, const MatView &v, int layout, int R, int CC);

namespace {

// ---------------------------------------------------------- tile shapes ---
// FP64 tile shapes (quaternion rows x columns); all use 4 warps.
constexpr int kNumShapes = 4;
__host__ __device__ constexpr int shape_m(int s) { return (s == 0 || s == 2) ? 32 : 16; }
__host__ __device__ constexpr int shape_n(int s) { return s < 2 ? 32 : 16; }

// Size buckets: m and n each fall in one of 5 ranges.
constexpr int kEdges[4] = {16, 32, 64, 128};
constexpr int kBuckets = 25;

int range_of(int64_t x) {
  int b = 0;
  while (b < 4 && x > kEdges[b]) ++b;
  return b;
}
int bucket_of(int64_t m, int64_t n) { return range_of(m) * 5 + range_of(n); }

std::mutex g_table_mu;
int g_table[kBuckets];
bool g_table_set = false;

// Default before tuning: per dimension the shape with the least padding.
int default_shape(int64_t m, int64_t n) {
  const int64_t pm16 = (m + 15) / 16 * 16, pm32 = (m + 31) / 32 * 32;
  const int64_t pn16 = (n + 15) / 16 * 16, pn32 = (n + 31) / 32 * 32;
  const bool sm = pm16 < pm32, sn = pn16 < pn32;
  if (sm && sn) return 3;
  if (sm) return 1;
  if (sn) return 2;
  return 0;
}

// Split-BF16 batches: column-tile width per size bucket (code 0: 64, 1: 32,
// 2: 16 quaternion columns), 64 before tuning.
constexpr int kSplitWidths = 3;
__host__ __device__ constexpr int split_width(int code) { return code == 1 ? 32 : (code == 2 ? 16 : 64); }
int g_split_table[kBuckets];
bool g_split_table_set = false;

int split_width_for(int64_t m, int64_t n) {
  std::lock_guard<std::mutex> lock(g_table_mu);
  if (!g_split_table_set) return 64;
  const int c = g_split_table[bucket_of(m, n)];
  return split_width(c >= 0 && c < kSplitWidths ? c : 0);
}

int shape_for(int64_t m, int64_t n) {
  std::lock_guard<std::mutex> lock(g_table_mu);
  if (!g_table_set) return default_shape(m, n);
  const int s = g_table[bucket_of(m, n)];
  return (s >= 0 && s < kNumShapes) ? s : default_shape(m, n);
}

// ------------------------------------------------------ device structs ---
struct alignas(128) GDesc64 {
  CUtensorMap tmA;
  CUtensorMap tmB;
  fp64::Operands op;
};

struct TileEntry {
  int32_t prob, tm, tn, code;  // code = shape | ta << 4 | tb << 5
};

constexpr size_t kHeaderBytes = 256;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ------------------------------------------------------------ kernels ---
template <int LAYOUT>
__global__ void __launch_bounds__(fp64::kThreads)
    grouped_fp64_kernel(const GDesc64 *__restrict__ descs, const TileEntry *__restrict__ tiles,
                        int ntiles, int *counter, uint64_t limit_ns) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double *sA = reinterpret_cast<double *>(smem_raw);
  double *sB = sA + fp64::kStages * fp64::kMaxTileElems;
  uint64_t *full = reinterpret_cast<uint64_t *>(sB + fp64::kStages * fp64::kMaxTileElems);
  __shared__ int s_next;
  if (threadIdx.x == 0) {
    for (int s = 0; s < fp64::kStages; ++s) mbar_init(&full[s], 1);
    fence_barrier_init();
  }
  __syncthreads();
  uint32_t kb_run = 0;
  while (true) {
    if (threadIdx.x == 0) s_next = atomicAdd(counter, 1);
    __syncthreads();
    const int t = s_next;
    __syncthreads();
    if (t >= ntiles) break;
    const TileEntry e = tiles[t];
    const GDesc64 *d = descs + e.prob;
    const int shape = e.code & 15;
    const int64_t i0 = static_cast<int64_t>(e.tm) * shape_m(shape);
    const int64_t n0 = static_cast<int64_t>(e.tn) * shape_n(shape);
    const CUtensorMap *ta = &d->tmA, *tb = &d->tmB;
    bool ok;
#define QG_TILE(S, TA, TB)                                                                   \
  ok = fp64::tile<LAYOUT, TA, TB, shape_m(S), shape_n(S)>(d->op, ta, tb, sA, sB, full, kb_run, \
                                                          i0, n0, limit_ns, &g_grouped_error)
    switch (e.code & 0x3F) {
      case 0x00: QG_TILE(0, false, false); break;
      case 0x10: QG_TILE(0, true, false); break;
      case 0x20: QG_TILE(0, false, true); break;
      case 0x30: QG_TILE(0, true, true); break;
      case 0x01: QG_TILE(1, false, false); break;
      case 0x11: QG_TILE(1, true, false); break;
      case 0x21: QG_TILE(1, false, true); break;
      case 0x31: QG_TILE(1, true, true); break;
      case 0x02: QG_TILE(2, false, false); break;
      case 0x12: QG_TILE(2, true, false); break;
      case 0x22: QG_TILE(2, false, true); break;
      case 0x32: QG_TILE(2, true, true); break;
      case 0x03: QG_TILE(3, false, false); break;
      case 0x13: QG_TILE(3, true, false); break;
      case 0x23: QG_TILE(3, false, true); break;
      default: QG_TILE(3, true, true); break;
    }
#undef QG_TILE
    if (!ok) break;
    // the next tile reuses the ring: every thread is past this tile's reads
    __syncthreads();
  }
}

// ------------------------------------------------------- split kernels ---
struct GroupedErr {
  static __device__ int *word() { return &g_grouped_error; }
};

// Pre-pass over the split operands of every problem: entry = (problem,
// is_b, row tile, k tile).  At most 40 registers, so 6 CTAs fit on an SM: the
// tiles are small and ragged, and more resident CTAs keep more loads in
// flight.  (Measured on GB300: double-buffering each CTA's tiles with
// cp.async at 5 CTAs per SM was slower, 1.68 against 1.56 ms on the
// 4096-problem batch.)
__global__ void __launch_bounds__(256, 6)
    grouped_prepass_kernel(const split::SplitProb *__restrict__ probs,
                           const int4 *__restrict__ ptiles, int n) {
  __shared__ float4 tile[32][33];
  for (int t = blockIdx.x; t < n; t += gridDim.x) {
    const int4 e = ptiles[t];
    if (e.y)
      split::prep_tile<true>(probs[e.x].pb, e.z, e.w, tile);
    else
      split::prep_tile<false>(probs[e.x].pa, e.z, e.w, tile);
    __syncthreads();
  }
}

// ---------------------------------------------------------- host plan ---
struct PlanLayout {
  size_t desc_off, tile_off, total;
  int64_t tiles;
};

int validate_problems(const qgemm_problem *problems, int64_t count, int layout, int precision,
                      std::vector<GemmDesc> *out) {
  if (count < 0) return -2;
  if (count > 0 && problems == nullptr) return -1;
  if (layout != QGEMM_INTERLEAVED && layout != QGEMM_SPLIT_PLANES) return -3;
  if (!precision_ok(precision)) return -4;
  out->resize(static_cast<size_t>(count));
  for (int64_t p = 0; p < count; ++p) {
    const qgemm_problem &q = problems[p];
    const int rc = validate_gemm(q.opA, q.opB, q.m, q.n, q.k, q.alpha, q.A, q.lda, q.psA, q.B,
                                 q.ldb, q.psB, q.beta, q.C, q.ldc, q.psC, layout, precision,
                                 &(*out)[static_cast<size_t>(p)]);
    if (rc) {
      const int64_t code = 1000 * (p + 1) - rc;  // rc < 0
      return code > 0x7fffffff ? -0x7fffffff : -static_cast<int>(code);
    }
  }
  return 0;
}

PlanLayout layout_fp64(const std::vector<GemmDesc> &ds) {
  PlanLayout L{};
  int64_t tiles = 0;
  for (const GemmDesc &d : ds) {
    if (d.m == 0 || d.n == 0) continue;
    const int s = shape_for(d.m, d.n);
    tiles += ((d.m + shape_m(s) - 1) / shape_m(s)) * ((d.n + shape_n(s) - 1) / shape_n(s));
  }
  L.tiles = tiles;
  L.desc_off = kHeaderBytes;
  L.tile_off = align_up(L.desc_off + ds.size() * sizeof(GDesc64), 256);
  L.total = align_up(L.tile_off + static_cast<size_t>(tiles) * sizeof(TileEntry), 256);
  return L;
}

int set_grouped_smem(int layout) {
  static bool done[2][64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return QGEMM_ERR_UNSUPPORTED;
  if (!done[layout][dev]) {
    cudaError_t e = layout == QGEMM_INTERLEAVED
                        ? cudaFuncSetAttribute(grouped_fp64_kernel<0>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(fp64::kSmemBytes))
                        : cudaFuncSetAttribute(grouped_fp64_kernel<1>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(fp64::kSmemBytes));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return QGEMM_ERR_CUDA;
    }
    done[layout][dev] = true;
  }
  return QGEMM_SUCCESS;
}

// ---- split precision ----
struct SplitLayout {
  size_t desc_off, tile_off, ptile_off, data_off, total;
  int64_t tiles, ptiles;
  std::vector<size_t> a_off, b_off;  // per problem, relative to the workspace
  std::vector<int64_t> kp;
  std::vector<int> width;            // per problem: column-tile width
};

int64_t split_kp(int64_t k) { return (k + 7) / 8 * 8; }

// Conjugate transpose of an op: (op(X))^H = op'(X).
int op_conjtrans(int op) {
  switch (op) {
    case QGEMM_OP_N: return QGEMM_OP_H;
    case QGEMM_OP_H: return QGEMM_OP_N;
    case QGEMM_OP_T: return QGEMM_OP_C;
    default: return QGEMM_OP_T;
  }
}

// MMA work of an m x n problem in split-BF16 tiles: rows padded to BM, every
// column tile to its MMA width (16-column granules, at most BNQ).
int64_t split_padded(int64_t m, int64_t n) {
  const int64_t rows = (m + split::BM - 1) / split::BM * split::BM;
  const int64_t full = n / split::BNQ * split::BNQ, rem = n % split::BNQ;
  return rows * (full + (rem + 15) / 16 * 16);
}

// (AB)^H = B^H A^H (Sec. 2.2): when it pads less, a problem is computed as
// D = op(B)^H op(A)^H and written back as C = conj(D)^T by the epilogue.
GemmDesc oriented(const GemmDesc &d, bool *swapped) {
  *swapped = d.k > 0 && split_padded(d.n, d.m) < split_padded(d.m, d.n);
  if (!*swapped) return d;
  GemmDesc t = d;
  t.m = d.n;
  t.n = d.m;
  t.opA = op_conjtrans(d.opB);
  t.opB = op_conjtrans(d.opA);
  t.A = d.B;
  t.B = d.A;
  t.swap = 1;
  return t;
}

SplitLayout layout_split(const std::vector<GemmDesc> &ds_in) {
  SplitLayout L{};
  int64_t tiles = 0, ptiles = 0;
  L.a_off.resize(ds_in.size());
  L.b_off.resize(ds_in.size());
  L.kp.resize(ds_in.size());
  L.width.assign(ds_in.size(), 64);
  size_t data = 0;
  for (size_t p = 0; p < ds_in.size(); ++p) {
    bool sw;
    const GemmDesc d = oriented(ds_in[p], &sw);
    L.kp[p] = split_kp(d.k);
    if (d.m == 0 || d.n == 0) continue;
    const int64_t w = L.width[p] = split_width_for(d.m, d.n);
    tiles += ((d.m + split::BM - 1) / split::BM) * ((d.n + w - 1) / w);
    if (d.k > 0) {
      const int64_t kt = (d.k + 31) / 32;
      ptiles += ((d.m + 31) / 32) * kt + ((d.n + 31) / 32) * kt;
      L.a_off[p] = data;
      data = align_up(data + static_cast<size_t>(split::TERMS) * split::PLANES * d.m * L.kp[p] * 2,
                      1024);
      L.b_off[p] = data;
      data = align_up(data + static_cast<size_t>(split::TERMS) * split::PLANES * d.n * L.kp[p] * 2,
                      1024);
    }
  }
  L.tiles = tiles;
  L.ptiles = ptiles;
  L.desc_off = kHeaderBytes;
  L.tile_off = align_up(L.desc_off + ds_in.size() * sizeof(split::SplitProb), 256);
  L.ptile_off = align_up(L.tile_off + static_cast<size_t>(tiles) * sizeof(int4), 256);
  L.data_off = align_up(L.ptile_off + static_cast<size_t>(ptiles) * sizeof(int4), 1024);
  for (size_t p = 0; p < ds_in.size(); ++p) {
    L.a_off[p] += L.data_off;
    L.b_off[p] += L.data_off;
  }
  L.total = L.data_off + data;
  return L;
}

int set_split_smem() {
  static bool done[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return QGEMM_ERR_UNSUPPORTED;
  if (!done[dev]) {
    if (cudaFuncSetAttribute(split::gemm_kernel<GroupedErr, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(split::kSmemBytes)) != cudaSuccess) {
      cudaGetLastError();
      return QGEMM_ERR_CUDA;
    }
    done[dev] = true;
  }
  return QGEMM_SUCCESS;
}

void double_float4(const double *x, float *hi, float *lo) {
  for (int s = 0; s < 4; ++s) {
    hi[s] = static_cast<float>(x[s]);
    lo[s] = static_cast<float>(x[s] - static_cast<double>(hi[s]));
  }
}

// Pre-pass arguments of one operand of a grouped problem: op(X) with `rows`
// op rows, scaled by s on the given side (kScale*).
void prep_args(split::PrepArgs &a, const MatView &v, int op, bool is_b, int64_t rows,
               int64_t k, int64_t kp, int layout, __nv_bfloat16 *out, int smode,
               const double *s) {
  a = split::PrepArgs{};
  a.X = static_cast<const float *>(v.ptr);
  a.ld = v.ld;
  a.ps = v.ps;
  a.rows = rows;
  a.kq = k;
  a.kp = kp;
  a.out = out;
  a.layout = layout;
  a.row_contig = is_b ? (op_trans(op) ? 1 : 0) : (op_trans(op) ? 0 : 1);
  a.conj = op_conj(op) ? 1 : 0;
  a.width = 4;
  a.planes = 4;
  a.smode = smode;
  if (s) double_float4(s, a.s_hi, a.s_lo);
}

int prepare_split(const std::vector<GemmDesc> &ds_in, int layout, unsigned char *ws,
                  size_t ws_bytes, cudaStream_t s, qgemm_grouped_plan *plan) {
  const SplitLayout L = layout_split(ds_in);
  if (ws_bytes < L.total) return -6;
  if (L.tiles > 0x7fffffff || L.ptiles > 0x7fffffff) return QGEMM_ERR_UNSUPPORTED;
  int rc = set_split_smem();
  if (rc) return rc;
  const size_t host_bytes = L.data_off - L.desc_off;
  std::vector<unsigned char> host(host_bytes, 0);
  auto *hd = reinterpret_cast<split::SplitProb *>(host.data());
  std::vector<int4> tiles, ptiles;
  std::vector<int> tile_kb;
  for (size_t p = 0; p < ds_in.size(); ++p) {
    bool sw;
    const GemmDesc d = oriented(ds_in[p], &sw);
    if (d.m == 0 || d.n == 0) continue;
    if (d.k > split::kMaxK) return QGEMM_ERR_UNSUPPORTED;
    split::SplitProb &q = hd[p];
    const int64_t kp = L.kp[p];
    auto *wa = reinterpret_cast<__nv_bfloat16 *>(ws + L.a_off[p]);
    auto *wb = reinterpret_cast<__nv_bfloat16 *>(ws + L.b_off[p]);
    q.g.m = d.m;
    q.g.n = d.n;
    q.g.num_kb = static_cast<int>(d.k > 0 ? (d.k + split::KQ - 1) / split::KQ : 0);
    q.g.num_mt = static_cast<int>((d.m + split::BM - 1) / split::BM);
    q.g.num_nt = static_cast<int>((d.n + split::BNQ - 1) / split::BNQ);
    q.g.pa = 4;
    q.g.pb = 4;
    q.g.layout = layout;
    q.g.beta_zero = d.beta_zero ? 1 : 0;
    q.g.beta_real = (d.beta[1] == 0.0 && d.beta[2] == 0.0 && d.beta[3] == 0.0) ? 1 : 0;
    q.g.c_vec4 = (reinterpret_cast<uintptr_t>(d.C) % 16 == 0) ? 1 : 0;
    q.g.C = static_cast<float *>(d.C);
    q.g.ldc = d.ldc;
    q.g.psC = d.psc;
    q.g.swap = sw ? 1 : 0;
    split::set_beta(q.g, d.beta);
    if (d.k > 0) {
      // alpha: on the left of op(A), or (turned around) conj(alpha) on the
      // right of op(A)^H, the B side: (alpha A B)^H = B^H (A^H conj(alpha))
      const double *al = d.alpha;
      const bool real = al[1] == 0.0 && al[2] == 0.0 && al[3] == 0.0;
      const int smode = (real && al[0] == 1.0) ? split::kScaleNone
                        : real                 ? split::kScaleReal
                        : sw                   ? split::kScaleRight
                                               : split::kScaleLeft;
      const double conj_al[4] = {al[0], -al[1], -al[2], -al[3]};
      prep_args(q.pa, d.A, d.opA, false, d.m, d.k, kp, layout, wa,
                sw ? split::kScaleNone : smode, al);
      prep_args(q.pb, d.B, d.opB, true, d.n, d.k, kp, layout, wb,
                sw ? smode : split::kScaleNone, conj_al);
      if (!encode_split_planes(&q.tmA, wa, d.k, kp, d.m, 4, split::BM) ||
          !encode_split_planes(&q.tmB, wb, d.k, kp, d.n, 4, split::BNQ))
        return QGEMM_ERR_UNSUPPORTED;
      const int kt = static_cast<int>((d.k + 31) / 32);
      for (int r = 0; r < (d.m + 31) / 32; ++r)
        for (int c = 0; c < kt; ++c) ptiles.push_back(make_int4(static_cast<int>(p), 0, r, c));
      for (int r = 0; r < (d.n + 31) / 32; ++r)
        for (int c = 0; c < kt; ++c) ptiles.push_back(make_int4(static_cast<int>(p), 1, r, c));
    }
    if (q.g.num_kb >= (1 << 24) || d.n > 0x7fffffff) return QGEMM_ERR_UNSUPPORTED;
    const int width = L.width[p];
    for (int a = 0; a < q.g.num_mt; ++a)
      for (int64_t n0 = 0; n0 < d.n; n0 += width) {
        // (problem, row tile, first column, stages | MMA width << 24): the
        // kernel needs no parameter load to start the tile
        const int64_t rem = d.n - n0;
        const int ncols = rem >= width ? width : static_cast<int>((rem + 15) / 16 * 16);
        tiles.push_back(make_int4(static_cast<int>(p), a, static_cast<int>(n0),
                                  q.g.num_kb | (ncols << 24)));
        tile_kb.push_back(q.g.num_kb);
      }
  }
  // longest tiles first; a problem's tiles stay adjacent (stable), so they run
  // at about the same time and share its operands in L2
  std::vector<int32_t> order(tiles.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = static_cast<int32_t>(i);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return tile_kb[a] > tile_kb[b]; });
  if (static_cast<int64_t>(tiles.size()) != L.tiles) return QGEMM_ERR_UNSUPPORTED;
  int4 *ht = reinterpret_cast<int4 *>(host.data() + (L.tile_off - L.desc_off));
  for (size_t i = 0; i < order.size(); ++i) ht[i] = tiles[order[i]];
  int4 *hp = reinterpret_cast<int4 *>(host.data() + (L.ptile_off - L.desc_off));
  for (size_t i = 0; i < ptiles.size(); ++i) hp[i] = ptiles[i];
  if (!host.empty() && cudaMemcpyAsync(ws + L.desc_off, host.data(), host.size(),
                                       cudaMemcpyHostToDevice, s) != cudaSuccess) {
    cudaGetLastError();
    return QGEMM_ERR_CUDA;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  plan->workspace_bytes = L.total;
  plan->tiles = L.tiles;
  plan->grid = static_cast<int32_t>(std::min<int64_t>(std::max<int64_t>(L.tiles, 1), sms));
  // pre-pass CTAs: up to 64 per SM (grid-stride beyond), 6 resident per SM
  plan->reserved0 = static_cast<int32_t>(
      std::min<int64_t>(std::max<int64_t>(L.ptiles, 1), static_cast<int64_t>(sms) * 64));
  plan->desc_offset = static_cast<int64_t>(L.desc_off);
  plan->tile_offset = static_cast<int64_t>(L.tile_off);
  plan->data_offset = static_cast<int64_t>(L.data_off);
  plan->reserved[0] = static_cast<int64_t>(L.ptile_off);
  plan->reserved[1] = L.ptiles;
  return QGEMM_SUCCESS;
}

int launch_split(const qgemm_grouped_plan *plan, cudaStream_t s) {
  unsigned char *ws = static_cast<unsigned char *>(plan->workspace);
  const auto *probs = reinterpret_cast<const split::SplitProb *>(ws + plan->desc_offset);
  const auto *tiles = reinterpret_cast<const int4 *>(ws + plan->tile_offset);
  const auto *ptiles = reinterpret_cast<const int4 *>(ws + plan->reserved[0]);
  const int np = static_cast<int>(plan->reserved[1]);
  if (np > 0) {
    grouped_prepass_kernel<<<plan->reserved0, 256, 0, s>>>(probs, ptiles, np);
    if (int rc_ = launch_status()) return rc_;
  }
  CUtensorMap none;
  std::memset(&none, 0, sizeof(none));
  split::GemmParams g{};
  split::gemm_kernel<GroupedErr, true><<<plan->grid, split::kThreads, split::kSmemBytes, s>>>(
      none, none, g, probs, tiles, static_cast<int>(plan->tiles), wait_limit_ns(), 0);
  return launch_status();
}

}  // namespace

int grouped_take_device_error() {
  int v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_grouped_error, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return QGEMM_ERR_CUDA;
  }
  cudaMemcpyToSymbol(g_grouped_error, &z, sizeof(int));
  return v;
}

}  // namespace qg

using namespace qg;

extern "C" {

size_t qgemm_grouped_workspace_bytes(const qgemm_problem *problems, int64_t count, int layout,
                                     int precision) {
  std::vector<GemmDesc> ds;
  if (validate_problems(problems, count, layout, precision, &ds)) return 0;
  if (precision == QGEMM_FP64) return layout_fp64(ds).total;
  if (precision == QGEMM_FP64_SLICED_BF16) return sliced_grouped_workspace_bytes(ds);
  return layout_split(ds).total;
}

int qgemm_grouped_prepare(const qgemm_problem *problems, int64_t count, int layout,
                          int precision, void *workspace, size_t workspace_bytes, void *stream,
                          qgemm_grouped_plan *plan) {
  if (plan == nullptr) return -8;
  std::memset(plan, 0, sizeof(*plan));
  std::vector<GemmDesc> ds;
  int rc = validate_problems(problems, count, layout, precision, &ds);
  if (rc) return rc;
  if (workspace == nullptr || reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return -5;
  if (precision != QGEMM_FP64) {
    rc = device_ready();
    if (rc) return rc;
    plan->workspace = workspace;
    plan->layout = layout;
    plan->precision = precision;
    plan->count = count;
    if (precision == QGEMM_FP64_SLICED_BF16)
      return prepare_sliced_grouped(ds, layout, static_cast<unsigned char *>(workspace),
                                    workspace_bytes, static_cast<cudaStream_t>(stream), plan);
    return prepare_split(ds, layout, static_cast<unsigned char *>(workspace), workspace_bytes,
                         static_cast<cudaStream_t>(stream), plan);
  }
  const PlanLayout L = layout_fp64(ds);
  if (workspace_bytes < L.total) return -6;
  if (L.tiles > 0x7fffffff) return QGEMM_ERR_UNSUPPORTED;
  rc = device_ready();
  if (rc) return rc;
  rc = set_grouped_smem(layout);  // here, so a captured launch needs no attribute call
  if (rc) return rc;

  std::vector<unsigned char> host(L.total - L.desc_off, 0);
  GDesc64 *hd = reinterpret_cast<GDesc64 *>(host.data());
  std::vector<TileEntry> tiles;
  tiles.reserve(static_cast<size_t>(L.tiles));
  std::vector<int64_t> tile_k;
  tile_k.reserve(static_cast<size_t>(L.tiles));
  for (size_t p = 0; p < ds.size(); ++p) {
    const GemmDesc &d = ds[p];
    GDesc64 &g = hd[p];
    if (d.m == 0 || d.n == 0) continue;
    const int s = shape_for(d.m, d.n);
    const bool ta = op_trans(d.opA), tb = op_trans(d.opB);
    g.op = fp64_operands(d);
    if (d.k > 0) {
      g.op.tmaA = encode_fp64_operand(&g.tmA, d.A, layout, ta ? fp64::kBKQ : shape_m(s),
                                      ta ? shape_m(s) : fp64::kBKQ) ? 1 : 0;
      g.op.tmaB = encode_fp64_operand(&g.tmB, d.B, layout, tb ? shape_n(s) : fp64::kBKQ,
                                      tb ? fp64::kBKQ : shape_n(s)) ? 1 : 0;
    }
    const int64_t tm_n = (d.m + shape_m(s) - 1) / shape_m(s);
    const int64_t tn_n = (d.n + shape_n(s) - 1) / shape_n(s);
    for (int64_t a = 0; a < tm_n; ++a)
      for (int64_t b = 0; b < tn_n; ++b) {
        tiles.push_back(TileEntry{static_cast<int32_t>(p), static_cast<int32_t>(a),
                                  static_cast<int32_t>(b), s | (ta << 4) | (tb << 5)});
        tile_k.push_back(d.k);
      }
  }
  // longest tiles first
  std::vector<int32_t> order(tiles.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = static_cast<int32_t>(i);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return tile_k[a] > tile_k[b]; });
  TileEntry *ht = reinterpret_cast<TileEntry *>(host.data() + (L.tile_off - L.desc_off));
  for (size_t i = 0; i < order.size(); ++i) ht[i] = tiles[order[i]];

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char *ws = static_cast<unsigned char *>(workspace);
  if (!host.empty() &&
      cudaMemcpyAsync(ws + L.desc_off, host.data(), host.size(), cudaMemcpyHostToDevice, s) !=
          cudaSuccess) {
    cudaGetLastError();
    return QGEMM_ERR_CUDA;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  plan->workspace = workspace;
  plan->workspace_bytes = L.total;
  plan->layout = layout;
  plan->precision = precision;
  plan->count = count;
  plan->tiles = L.tiles;
  plan->grid = static_cast<int32_t>(std::min<int64_t>(std::max<int64_t>(L.tiles, 1), 2 * sms));
  plan->desc_offset = static_cast<int64_t>(L.desc_off);
  plan->tile_offset = static_cast<int64_t>(L.tile_off);
  plan->data_offset = static_cast<int64_t>(L.total);
  return QGEMM_SUCCESS;
}

int qgemm_grouped_launch(const qgemm_grouped_plan *plan, void *stream) {
  if (plan == nullptr || plan->workspace == nullptr) return -1;
  if (plan->tiles == 0) return QGEMM_SUCCESS;
  int rc = device_ready();
  if (rc) return rc;
  if (plan->precision == QGEMM_FP64_SLICED_BF16)
    return launch_sliced_grouped(plan, static_cast<cudaStream_t>(stream));
  if (plan->precision == QGEMM_FP32_SPLIT_BF16)
    return launch_split(plan, static_cast<cudaStream_t>(stream));
  rc = set_grouped_smem(plan->layout);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char *ws = static_cast<unsigned char *>(plan->workspace);
  int *counter = reinterpret_cast<int *>(ws);
  if (cudaMemsetAsync(counter, 0, sizeof(int), s) != cudaSuccess) {
    cudaGetLastError();
    return QGEMM_ERR_CUDA;
  }
  const GDesc64 *descs = reinterpret_cast<const GDesc64 *>(ws + plan->desc_offset);
  const TileEntry *tiles = reinterpret_cast<const TileEntry *>(ws + plan->tile_offset);
  const int nt = static_cast<int>(plan->tiles);
  if (plan->layout == QGEMM_INTERLEAVED)
    grouped_fp64_kernel<0><<<plan->grid, fp64::kThreads, fp64::kSmemBytes, s>>>(
        descs, tiles, nt, counter, wait_limit_ns());
  else
    grouped_fp64_kernel<1><<<plan->grid, fp64::kThreads, fp64::kSmemBytes, s>>>(
        descs, tiles, nt, counter, wait_limit_ns());
  return launch_status();
}

int qgemm_batched_grouped(const qgemm_problem *problems, int64_t count, int layout,
                          int precision, void *workspace, size_t workspace_bytes, void *stream) {
  qgemm_grouped_plan plan;
  const int rc = qgemm_grouped_prepare(problems, count, layout, precision, workspace,
                                       workspace_bytes, stream, &plan);
  if (rc) return rc;
  return qgemm_grouped_launch(&plan, stream);
}

int qgemm_grouped_set_tile_table(int precision, const int32_t *table, int32_t entries) {
  if (precision != QGEMM_FP64 && precision != QGEMM_FP32_SPLIT_BF16) return -1;
  if (table != nullptr && entries != kBuckets) return -3;
  const bool split = precision == QGEMM_FP32_SPLIT_BF16;
  std::lock_guard<std::mutex> lock(g_table_mu);
  if (table == nullptr) {
    (split ? g_split_table_set : g_table_set) = false;
    return QGEMM_SUCCESS;
  }
  const int limit = split ? kSplitWidths : kNumShapes;
  for (int i = 0; i < kBuckets; ++i)
    if (table[i] < 0 || table[i] >= limit) return -2;
  std::memcpy(split ? g_split_table : g_table, table, sizeof(g_table));
  (split ? g_split_table_set : g_table_set) = true;
  return QGEMM_SUCCESS;
}

int qgemm_grouped_tile_info(int32_t *num_shapes, int32_t *rows, int32_t *cols,
                            int32_t *num_buckets, int32_t *edges) {
  if (num_shapes) *num_shapes = kNumShapes;
  if (num_buckets) *num_buckets = kBuckets;
  for (int i = 0; i < kNumShapes; ++i) {
    if (rows) rows[i] = shape_m(i);
    if (cols) cols[i] = shape_n(i);
  }
  for (int i = 0; i < 4 && edges; ++i) edges[i] = kEdges[i];
  return QGEMM_SUCCESS;
}

}  // extern "C"
