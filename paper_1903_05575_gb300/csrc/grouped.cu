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
// is_b, row tile, k tile).  At most 32 registers, so 8 CTAs fit on an SM: the
// tiles are small and ragged, and more resident CTAs keep more loads in flight.
__global__ void __launch_bounds__(256, 8)
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
};

int64_t split_kp(int64_t k) { return ((4 * k + split::BK - 1) / split::BK) * split::BK; }

// Conjugate transpose of an op: (op(X))^H = op'(X).
int op_conjtrans(int op) {
  switch (op) {
    case QGEMM_OP_N: return QGEMM_OP_H;
    case QGEMM_OP_H: return QGEMM_OP_N;
    case QGEMM_OP_T: return QGEMM_OP_C;
    default: return QGEMM_OP_T;
  }
}

// (AB)^H = B^H A^H (Sec. 2.2): when it pads less (tile rows are padded to
// 128, columns to 64), a problem is computed as D = op(B)^H op(A)^H and
// written back as C = conj(D)^T by the epilogue.
GemmDesc oriented(const GemmDesc &d, bool *swapped) {
  const int64_t pad_n = ((d.m + split::BM - 1) / split::BM) * split::BM *
                        (((d.n + split::BNQ - 1) / split::BNQ) * split::BNQ);
  const int64_t pad_s = ((d.n + split::BM - 1) / split::BM) * split::BM *
                        (((d.m + split::BNQ - 1) / split::BNQ) * split::BNQ);
  *swapped = d.k > 0 && pad_s < pad_n && std::getenv("QGEMM_GROUPED_NO_SWAP") == nullptr;
  if (!*swapped) return d;
  GemmDesc t = d;
  t.m = d.n;
  t.n = d.m;
  t.opA = op_conjtrans(d.opB);
  t.opB = op_conjtrans(d.opA);
  t.A = d.B;
  t.B = d.A;
  return t;
}

SplitLayout layout_split(const std::vector<GemmDesc> &ds_in) {
  std::vector<GemmDesc> ds(ds_in.size());
  for (size_t p = 0; p < ds_in.size(); ++p) {
    bool sw;
    ds[p] = oriented(ds_in[p], &sw);
  }
  SplitLayout L{};
  int64_t tiles = 0, ptiles = 0;
  L.a_off.resize(ds.size());
  L.b_off.resize(ds.size());
  L.kp.resize(ds.size());
  size_t data = 0;
  for (size_t p = 0; p < ds.size(); ++p) {
    const GemmDesc &d = ds[p];
    L.kp[p] = split_kp(d.k);
    if (d.m == 0 || d.n == 0) continue;
    tiles += ((d.m + split::BM - 1) / split::BM) * ((d.n + split::BNQ - 1) / split::BNQ);
    if (d.k > 0) {
      const int64_t kt = (L.kp[p] / 4 + 31) / 32;
      ptiles += ((d.m + 31) / 32) * kt + ((d.n + 31) / 32) * kt;
      L.a_off[p] = data;
      data = align_up(data + static_cast<size_t>(split::TERMS) * d.m * L.kp[p] * 2, 1024);
      L.b_off[p] = data;
      data = align_up(data + static_cast<size_t>(split::TERMS) * 4 * d.n * L.kp[p] * 2, 1024);
    }
  }
  L.tiles = tiles;
  L.ptiles = ptiles;
  L.desc_off = kHeaderBytes;
  L.tile_off = align_up(L.desc_off + ds.size() * sizeof(split::SplitProb), 256);
  L.ptile_off = align_up(L.tile_off + static_cast<size_t>(tiles) * sizeof(int4), 256);
  L.data_off = align_up(L.ptile_off + static_cast<size_t>(ptiles) * sizeof(int4), 1024);
  for (size_t p = 0; p < ds.size(); ++p) {
    L.a_off[p] += L.data_off;
    L.b_off[p] += L.data_off;
  }
  L.total = L.data_off + data;
  return L;
}

bool encode_split_map(CUtensorMap *map, const void *base, int64_t kp, int64_t rows, int box) {
  EncodeTiledFn enc = encode_tiled_fn();
  if (!enc || rows <= 0) return false;
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(kp), static_cast<cuuint64_t>(rows), split::TERMS};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(kp) * 2,
                           static_cast<cuuint64_t>(kp) * 2 * static_cast<cuuint64_t>(rows)};
  cuuint32_t boxd[3] = {split::BK, static_cast<cuuint32_t>(box), split::TERMS};
  cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides,
             boxd, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
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

int prepare_split(const std::vector<GemmDesc> &ds_in, int layout, unsigned char *ws,
                  size_t ws_bytes, cudaStream_t s, qgemm_grouped_plan *plan) {
  const SplitLayout L = layout_split(ds_in);
  std::vector<GemmDesc> ds(ds_in.size());
  std::vector<int> swapped(ds_in.size(), 0);
  for (size_t p = 0; p < ds_in.size(); ++p) {
    bool sw;
    ds[p] = oriented(ds_in[p], &sw);
    swapped[p] = sw ? 1 : 0;
  }
  if (ws_bytes < L.total) return -6;
  if (L.tiles > 0x7fffffff || L.ptiles > 0x7fffffff) return QGEMM_ERR_UNSUPPORTED;
  int rc = set_split_smem();
  if (rc) return rc;
  const size_t host_bytes = L.data_off - L.desc_off;
  std::vector<unsigned char> host(host_bytes, 0);
  auto *hd = reinterpret_cast<split::SplitProb *>(host.data());
  std::vector<int4> tiles, ptiles;
  std::vector<int> tile_kb;
  for (size_t p = 0; p < ds.size(); ++p) {
    const GemmDesc &d = ds[p];
    if (d.m == 0 || d.n == 0) continue;
    split::SplitProb &q = hd[p];
    const int64_t kp = L.kp[p];
    auto *wa = reinterpret_cast<__nv_bfloat16 *>(ws + L.a_off[p]);
    auto *wb = reinterpret_cast<__nv_bfloat16 *>(ws + L.b_off[p]);
    q.g.m = d.m;
    q.g.n = d.n;
    q.g.num_kb = static_cast<int>(d.k > 0 ? kp / split::BK : 0);
    q.g.num_mt = static_cast<int>((d.m + split::BM - 1) / split::BM);
    q.g.num_nt = static_cast<int>((d.n + split::BNQ - 1) / split::BNQ);
    q.g.layout = layout;
    q.g.beta_zero = d.beta_zero ? 1 : 0;
    q.g.c_vec4 = (reinterpret_cast<uintptr_t>(d.C) % 16 == 0) ? 1 : 0;
    q.g.C = static_cast<float *>(d.C);
    q.g.ldc = d.ldc;
    q.g.psC = d.psc;
    q.g.swap = swapped[p];
    for (int c = 0; c < 4; ++c) {
      q.g.alpha[c] = static_cast<float>(d.alpha[c]);
      q.g.beta[c] = static_cast<float>(d.beta[c]);
    }
    if (d.k > 0) {
      auto prep = [&](split::PrepArgs &a, const MatView &v, int op, bool is_b, int64_t rows,
                      __nv_bfloat16 *out) {
        a.X = static_cast<const float *>(v.ptr);
        a.ld = v.ld;
        a.ps = v.ps;
        a.rows = rows;
        a.kq = d.k;
        a.kp = kp;
        a.term_stride = (is_b ? 4 * rows : rows) * kp;
        a.out = out;
        a.layout = layout;
        a.row_contig = is_b ? (op_trans(op) ? 1 : 0) : (op_trans(op) ? 0 : 1);
        a.negmask = op_conj(op) ? 0xEu : 0u;
        a.width = 4;
        a.kw = 4;
      };
      prep(q.pa, d.A, d.opA, false, d.m, wa);
      prep(q.pb, d.B, d.opB, true, d.n, wb);
      if (!encode_split_map(&q.tmA, wa, kp, d.m, split::BM) ||
          !encode_split_map(&q.tmB, wb, kp, 4 * d.n, split::BN))
        return QGEMM_ERR_UNSUPPORTED;
      const int kt = static_cast<int>((kp / 4 + 31) / 32);
      for (int r = 0; r < (d.m + 31) / 32; ++r)
        for (int c = 0; c < kt; ++c) ptiles.push_back(make_int4(static_cast<int>(p), 0, r, c));
      for (int r = 0; r < (d.n + 31) / 32; ++r)
        for (int c = 0; c < kt; ++c) ptiles.push_back(make_int4(static_cast<int>(p), 1, r, c));
    }
    for (int a = 0; a < q.g.num_mt; ++a)
      for (int b = 0; b < q.g.num_nt; ++b) {
        tiles.push_back(make_int4(static_cast<int>(p), a, b, 0));
        tile_kb.push_back(q.g.num_kb);
      }
  }
  std::vector<int32_t> order(tiles.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = static_cast<int32_t>(i);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return tile_kb[a] > tile_kb[b]; });
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
  // pre-pass CTAs: up to 64 per SM (grid-stride beyond), 8 resident per SM
  plan->reserved0 = static_cast<int32_t>(
      std::min<int64_t>(std::max<int64_t>(L.ptiles, 1), static_cast<int64_t>(sms) * 64));
  plan->desc_offset = static_cast<int64_t>(L.desc_off);
  plan->tile_offset = static_cast<int64_t>(L.tile_off);
  plan->data_offset = static_cast<int64_t>(L.data_off);
  plan->reserved[0] = static_cast<int64_t>(L.ptile_off);
  plan->reserved[1] = L.ptiles;
  return QGEMM_SUCCESS;
}

// ---- split precision, fused (no operand workspace) ----
}  // namespace

// 3-D FP32 tensor map of a stored operand for a box of R x CC stored elements
// (component x row x column interleaved; row x column x plane for planes).
bool encode_fp32_operand(CUtensorMap *map, const MatView &v, int layout, int R, int CC) {
  const uintptr_t base = reinterpret_cast<uintptr_t>(v.ptr);
  if (base % 16 != 0 || v.rows <= 0 || v.cols <= 0) return false;
  cuuint64_t dims[3], strides[2];
  cuuint32_t box[3], estr[3] = {1, 1, 1};
  if (layout == QGEMM_INTERLEAVED) {
    dims[0] = 4;
    dims[1] = static_cast<cuuint64_t>(v.rows);
    dims[2] = static_cast<cuuint64_t>(v.cols);
    strides[0] = 16;
    strides[1] = static_cast<cuuint64_t>(v.ld) * 16;
    box[0] = 4;
    box[1] = R;
    box[2] = CC;
  } else {
    if (v.ld % 4 != 0 || v.ps % 4 != 0) return false;
    dims[0] = static_cast<cuuint64_t>(v.rows);
    dims[1] = static_cast<cuuint64_t>(v.cols);
    dims[2] = 4;
    strides[0] = static_cast<cuuint64_t>(v.ld) * 4;
    strides[1] = static_cast<cuuint64_t>(v.ps) * 4;
    box[0] = R;
    box[1] = CC;
    box[2] = 4;
  }
  if (dims[0] >= (1ull << 32) || dims[1] >= (1ull << 32) || dims[2] >= (1ull << 32)) return false;
  if (strides[0] >= (1ull << 40) || strides[1] >= (1ull << 40)) return false;
  EncodeTiledFn enc = encode_tiled_fn();
  if (!enc) return false;
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(v.ptr), dims, strides,
             box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace {

struct FusedLayout {
  size_t desc_off, tile_off, total;
  int64_t tiles;
};

FusedLayout layout_fused(const std::vector<GemmDesc> &ds) {
  FusedLayout L{};
  int64_t tiles = 0;
  for (const GemmDesc &d : ds)
    if (d.m > 0 && d.n > 0)
      tiles += ((d.m + split::BM - 1) / split::BM) * ((d.n + split::BNQ - 1) / split::BNQ);
  L.tiles = tiles;
  L.desc_off = kHeaderBytes;
  L.tile_off = align_up(L.desc_off + ds.size() * sizeof(split::FusedProb), 256);
  L.total = align_up(L.tile_off + static_cast<size_t>(tiles) * sizeof(int4), 256);
  return L;
}

// Fills the fused descriptors; false if some operand cannot be read by TMA.
bool fused_descs(const std::vector<GemmDesc> &ds, int layout, split::FusedProb *hd) {
  for (size_t p = 0; p < ds.size(); ++p) {
    const GemmDesc &d = ds[p];
    if (d.m == 0 || d.n == 0) continue;
    split::FusedProb &q = hd[p];
    const bool ta = op_trans(d.opA), tb = op_trans(d.opB);
    q.o.layout = layout;
    q.o.ta = ta ? 1 : 0;
    q.o.tb = tb ? 1 : 0;
    q.o.conj_a = op_conj(d.opA) ? 0xEu : 0u;
    q.o.conj_b = op_conj(d.opB) ? 0xEu : 0u;
    q.g.m = d.m;
    q.g.n = d.n;
    q.g.num_kb = static_cast<int>((d.k + split::FKQ - 1) / split::FKQ);
    q.g.num_mt = static_cast<int>((d.m + split::BM - 1) / split::BM);
    q.g.num_nt = static_cast<int>((d.n + split::BNQ - 1) / split::BNQ);
    q.g.layout = layout;
    q.g.beta_zero = d.beta_zero ? 1 : 0;
    q.g.c_vec4 = (reinterpret_cast<uintptr_t>(d.C) % 16 == 0) ? 1 : 0;
    q.g.C = static_cast<float *>(d.C);
    q.g.ldc = d.ldc;
    q.g.psC = d.psc;
    for (int c = 0; c < 4; ++c) {
      q.g.alpha[c] = static_cast<float>(d.alpha[c]);
      q.g.beta[c] = static_cast<float>(d.beta[c]);
    }
    if (d.k > 0) {
      if (!encode_fp32_operand(&q.tmA, d.A, layout, ta ? split::FKQ : split::BM,
                               ta ? split::BM : split::FKQ))
        return false;
      if (!encode_fp32_operand(&q.tmB, d.B, layout, tb ? split::BNQ : split::FKQ,
                               tb ? split::FKQ : split::BNQ))
        return false;
    }
  }
  return true;
}

int set_fused_smem() {
  static bool done[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return QGEMM_ERR_UNSUPPORTED;
  if (!done[dev]) {
    if (cudaFuncSetAttribute(split::fused_kernel<GroupedErr, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(split::kFusedSmemBytes)) != cudaSuccess) {
      cudaGetLastError();
      return QGEMM_ERR_CUDA;
    }
    done[dev] = true;
  }
  return QGEMM_SUCCESS;
}

// Returns QGEMM_ERR_UNSUPPORTED (before touching the workspace) when some
// operand is not TMA-addressable; the caller then takes the pre-pass path.
int prepare_fused(const std::vector<GemmDesc> &ds, int layout, unsigned char *ws,
                  size_t ws_bytes, cudaStream_t s, qgemm_grouped_plan *plan) {
  const FusedLayout L = layout_fused(ds);
  if (L.tiles > 0x7fffffff) return QGEMM_ERR_UNSUPPORTED;
  std::vector<unsigned char> host(L.total - L.desc_off, 0);
  auto *hd = reinterpret_cast<split::FusedProb *>(host.data());
  if (!fused_descs(ds, layout, hd)) return QGEMM_ERR_UNSUPPORTED;
  if (ws_bytes < L.total) return -6;
  int rc = set_fused_smem();
  if (rc) return rc;
  std::vector<int4> tiles;
  std::vector<int> tile_kb;
  for (size_t p = 0; p < ds.size(); ++p) {
    const GemmDesc &d = ds[p];
    if (d.m == 0 || d.n == 0) continue;
    for (int a = 0; a < hd[p].g.num_mt; ++a)
      for (int b = 0; b < hd[p].g.num_nt; ++b) {
        tiles.push_back(make_int4(static_cast<int>(p), a, b, 0));
        tile_kb.push_back(hd[p].g.num_kb);
      }
  }
  std::vector<int32_t> order(tiles.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = static_cast<int32_t>(i);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return tile_kb[a] > tile_kb[b]; });
  int4 *ht = reinterpret_cast<int4 *>(host.data() + (L.tile_off - L.desc_off));
  for (size_t i = 0; i < order.size(); ++i) ht[i] = tiles[order[i]];
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
  plan->desc_offset = static_cast<int64_t>(L.desc_off);
  plan->tile_offset = static_cast<int64_t>(L.tile_off);
  plan->data_offset = static_cast<int64_t>(L.total);
  plan->reserved[2] = 1;  // fused
  return QGEMM_SUCCESS;
}

int launch_fused(const qgemm_grouped_plan *plan, cudaStream_t s) {
  unsigned char *ws = static_cast<unsigned char *>(plan->workspace);
  const auto *probs = reinterpret_cast<const split::FusedProb *>(ws + plan->desc_offset);
  const auto *tiles = reinterpret_cast<const int4 *>(ws + plan->tile_offset);
  CUtensorMap none;
  std::memset(&none, 0, sizeof(none));
  split::GemmParams g{};
  split::FusedOps o{};
  const char *env = std::getenv("QGEMM_SPLIT_CHUNK");
  const int chunk = (env && std::atoi(env) > 0) ? std::atoi(env) : 2;
  split::fused_kernel<GroupedErr, true>
      <<<plan->grid, split::kFusedThreads, split::kFusedSmemBytes, s>>>(
          none, none, g, o, probs, tiles, static_cast<int>(plan->tiles), chunk, wait_limit_ns());
  return launch_status();
}

// The fused path is opt-in (QGEMM_GROUPED_FUSED=1): measured on GB300 its two
// converter warps limit it below the pre-pass path (4096-problem batch 26.7 vs
// 47.9 TFLOP/s), and more converter warps do not fit the register budget.
bool fused_enabled() {
  const char *e = std::getenv("QGEMM_GROUPED_FUSED");
  return e && e[0] == '1';
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
  const char *env = std::getenv("QGEMM_SPLIT_CHUNK");
  const int chunk = (env && std::atoi(env) > 0) ? std::atoi(env) : 2;
  split::gemm_kernel<GroupedErr, true><<<plan->grid, split::kThreads, split::kSmemBytes, s>>>(
      none, none, g, probs, tiles, static_cast<int>(plan->tiles), chunk, wait_limit_ns());
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
  if (fused_enabled()) {
    std::vector<unsigned char> probe(ds.size() * sizeof(split::FusedProb), 0);
    if (fused_descs(ds, layout, reinterpret_cast<split::FusedProb *>(probe.data())))
      return layout_fused(ds).total;
  }
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
    if (fused_enabled()) {
      rc = prepare_fused(ds, layout, static_cast<unsigned char *>(workspace), workspace_bytes,
                         static_cast<cudaStream_t>(stream), plan);
      if (rc != QGEMM_ERR_UNSUPPORTED) return rc;
    }
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
    return plan->reserved[2] == 1 ? launch_fused(plan, static_cast<cudaStream_t>(stream))
                                  : launch_split(plan, static_cast<cudaStream_t>(stream));
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
  if (precision != QGEMM_FP64) return -1;
  if (table != nullptr && entries != kBuckets) return -3;
  std::lock_guard<std::mutex> lock(g_table_mu);
  if (table == nullptr) {
    g_table_set = false;
    return QGEMM_SUCCESS;
  }
  for (int i = 0; i < kBuckets; ++i)
    if (table[i] < 0 || table[i] >= kNumShapes) return -2;
  std::memcpy(g_table, table, sizeof(g_table));
  g_table_set = true;
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
