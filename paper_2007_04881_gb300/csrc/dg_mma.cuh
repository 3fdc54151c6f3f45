// dg_mma.cuh -- row kernels whose local contractions A = U^T V run on the
// tensor cores (warp-level mma.sync), in two forms:
//   split-BF16: x = hi + lo with hi = bf16(x), lo = bf16(x - hi); each
//     product is hi*hi + hi*lo + lo*hi (the lo*lo term dropped), m16n8k16,
//     FP32 accumulation;
//   3xTF32: the same split with TF32 halves, m16n8k8, FP32 accumulation.
// Geometry, quadrature points and weights, basis values and the per-point
// rows are the FP32 form's (geometry records equal to the rounded FP64
// ones); only the
// contractions change.  The tensor cores' FP32 accumulation is not rounded
// to nearest at every addition, so its accumulators live for one chunk of
// points only and are added to IEEE FP32 running sums after each chunk:
// large elements (thousands of points) then keep the FP32 form's accuracy.
// Block rows are owned by warps exactly as in
// row_kernel: the diagonal block (volume + own faces, fixed order), the load
// vector and the off-diagonal blocks of an element are written once by the
// warp that owns it, with no atomics.
//
// Staging.  For an element, the rows of a chunk of C points are stored
// term-major (row t*C + c = term t of point c) with the dofs along the row:
// U[row][i] (own basis rows, 16*MT columns) and V[row][j] (the weighted
// test rows, NW columns; column N carries the load-vector weights R, so
// the load vector comes out of the same product as column N of U^T V).
// split-BF16 stores hi and lo planes and feeds the MMAs with ldmatrix.trans;
// 3xTF32 stores FP32 and splits while building the fragments.  BF16 rows
// of 2 or 4 16-byte units are XOR-swizzled (unit u of row r stored at
// u ^ f(r)), which keeps the 8 rows of every ldmatrix phase and of every
// staging-store phase on distinct banks without padding; other widths are
// padded to an odd number of units.  FP32 rows are padded to 8 or 24 mod 32
// words (conflict-free fragment loads) and their 16-byte units swizzled by
// bit 2 of the row (conflict-free staging stores).
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

#include "dg_device.cuh"

namespace dg {

enum : int { kMmaBf16 = 1, kMmaTf32 = 2 };

template <int D, int P, int K>
struct MmaCfg {
  static constexpr int N = nbasis(D, P);
  static constexpr int MT = (N + 15) / 16;             // 16-row tiles of the own dofs
  static constexpr int NW = (N + 1 + 15) / 16 * 16;    // staged columns of V: dofs + load column
  static constexpr int NT8 = (N + 1 + 7) / 8;          // 8-column tiles of the diagonal phases
  static constexpr int NTA = NW / 8;                   // 8-column tiles held in registers
  static constexpr int NTV = D + 1;                    // rows (terms) of a volume point
  static constexpr int C = 16;                         // points per element per chunk
  static constexpr int RW = C * NTV;                   // staged rows per element
  static constexpr int WU = 2 * MT, WV = NW / 8;      // 16-byte units of a BF16 row
  // swizzle (BF16: row width in units, 0 = padded instead; FP32: 1)
  static constexpr int ZU = K == kMmaBf16 ? ((WU == 2 || WU == 4) ? WU : 0) : 1;
  static constexpr int ZV = K == kMmaBf16 ? ((WV == 2 || WV == 4) ? WV : 0) : 1;
  static constexpr int SU = K == kMmaBf16 && ZU ? 16 * MT : 16 * MT + 8;  // row strides, elements
  static constexpr int SV = K == kMmaBf16 && ZV ? NW : NW + 8;
  static constexpr int ESZ = K == kMmaBf16 ? 2 : 4;
  static constexpr int NPL = K == kMmaBf16 ? 2 : 1;    // planes (hi, lo) or one FP32 plane
  static constexpr size_t per_elem = (size_t)RW * (SU + SV) * ESZ * NPL;
  static constexpr int G = per_elem <= 10 * 1024 ? 2 : 1;  // elements per warp
  static constexpr int KS = K == kMmaBf16 ? 16 : 8;         // rows per MMA k-step
  static constexpr int MINB = G == 2 ? 4 : 2;               // CTAs per SM the registers must allow
  static constexpr int PT = 4 * D + 5, PI = 17;
  static constexpr int QT = ipow_c(P + 2, D);
  static constexpr int NMAXC = nbasis(D, D == 2 ? kPMax2 : kPMax3);
  static constexpr size_t u_plane = (size_t)G * RW * SU;  // elements per plane
  static constexpr size_t v_plane = (size_t)G * RW * SV;
  static constexpr size_t stage_bytes = (u_plane + v_plane) * ESZ * NPL;
  static constexpr size_t head_bytes = align_up(sizeof(float) * (QT * (D + 1) + NMAXC), 16);
  static constexpr size_t warp_bytes =
      stage_bytes + align_up(sizeof(float) * G * PT, 16) + align_up(sizeof(int) * G * PI, 16);
  static constexpr size_t total = head_bytes + kWarps * warp_bytes;
  static_assert(RW % 16 == 0 && (2 * C) % 16 == 0, "chunk rows must fill whole k-steps");
  static_assert((SU * ESZ) % 16 == 0 && (SV * ESZ) % 16 == 0, "rows must stay 16-byte aligned");
};

// ---------------------------------------------------------------------------
// fragments
// ---------------------------------------------------------------------------

// XOR swizzle of the 16-byte units of a row (BF16 rows: Z units per row;
// Z = 1: the FP32 rows' swizzle; 0: none)
template <int Z>
__device__ __forceinline__ int swz(int row) {
  if constexpr (Z == 1 || Z == 2) return (row >> 2) & 1;
  if constexpr (Z == 4) return (row >> 1) & 3;
  return 0;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p))
               : "memory");
}

__device__ __forceinline__ void ldsm_x2_t(uint32_t (&r)[2], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(smem_u32(p))
               : "memory");
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void mma_tf32_1688(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(x - __uint_as_float(hi));
}

// pack (x0, x1) into bf16x2 hi and lo words (x0 in the low half)
__device__ __forceinline__ void split_bf16x2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// ---------------------------------------------------------------------------
// staging: one row of NC columns (multiple of 8): v[0..NV) then `extra` at
// column NV (when NV < NC), zeros after
// ---------------------------------------------------------------------------

template <int K, int S, int Z, int NC, int NV>
__device__ __forceinline__ void put_row(unsigned char* plane, size_t plane_elems, int row, const float* v,
                                        float extra) {
  auto val = [&](int j) -> float { return j < NV ? v[j < NV ? j : 0] : (j == NV ? extra : 0.f); };
  if constexpr (K == kMmaBf16) {
    __nv_bfloat16* hi = reinterpret_cast<__nv_bfloat16*>(plane) + (size_t)row * S;
    __nv_bfloat16* lo = hi + plane_elems;
#pragma unroll
    for (int q = 0; q < NC / 8; ++q) {
      uint32_t h[4], l[4];
#pragma unroll
      for (int w = 0; w < 4; ++w) split_bf16x2(val(8 * q + 2 * w), val(8 * q + 2 * w + 1), h[w], l[w]);
      const int u = q ^ swz<Z>(row);
      reinterpret_cast<uint4*>(hi)[u] = make_uint4(h[0], h[1], h[2], h[3]);
      reinterpret_cast<uint4*>(lo)[u] = make_uint4(l[0], l[1], l[2], l[3]);
    }
  } else {
    float* f = reinterpret_cast<float*>(plane) + (size_t)row * S;
#pragma unroll
    for (int q = 0; q < NC / 4; ++q)
      reinterpret_cast<float4*>(f)[q ^ swz<Z>(row)] =
          make_float4(val(4 * q), val(4 * q + 1), val(4 * q + 2), val(4 * q + 3));
  }
}

template <int K, int S, int NC>
__device__ __forceinline__ void zero_row(unsigned char* plane, size_t plane_elems, int row) {
  if constexpr (K == kMmaBf16) {
    __nv_bfloat16* hi = reinterpret_cast<__nv_bfloat16*>(plane) + (size_t)row * S;
#pragma unroll
    for (int q = 0; q < NC / 8; ++q) {
      reinterpret_cast<uint4*>(hi)[q] = make_uint4(0, 0, 0, 0);
      reinterpret_cast<uint4*>(hi + plane_elems)[q] = make_uint4(0, 0, 0, 0);
    }
  } else {
    float* f = reinterpret_cast<float*>(plane) + (size_t)row * S;
#pragma unroll
    for (int q = 0; q < NC / 4; ++q) reinterpret_cast<float4*>(f)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

template <int K, int S, int Z>
__device__ __forceinline__ void put_one(unsigned char* plane, size_t plane_elems, int row, int j, float x) {
  if constexpr (K == kMmaBf16) {
    __nv_bfloat16* hi =
        reinterpret_cast<__nv_bfloat16*>(plane) + (size_t)row * S + (((j >> 3) ^ swz<Z>(row)) << 3) + (j & 7);
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[0] = h;
    hi[plane_elems] = __float2bfloat16_rn(x - __bfloat162float(h));
  } else {
    reinterpret_cast<float*>(plane)[(size_t)row * S + (((j >> 2) ^ swz<Z>(row)) << 2) + (j & 3)] = x;
  }
}

// ---------------------------------------------------------------------------
// one k-step: acc[mi][nj] += U[k0 .. k0+KS)^T V[k0 .. k0+KS) for the 8-column
// tiles nj in [jt0, jt1) (warp-uniform range)
// ---------------------------------------------------------------------------

// acc takes hi*hi, accx the two cross products (two shorter dependency chains)
template <int K, int MT, int NTA, int SU, int SV, int ZU, int ZV>
__device__ __forceinline__ void mma_kstep(const unsigned char* Up, size_t u_plane, const unsigned char* Vp,
                                          size_t v_plane, int k0, int jt0, int jt1, float (&acc)[MT][NTA][4],
                                          float (&accx)[MT][NTA][4]) {
  const int lane = threadIdx.x & 31;
  if constexpr (K == kMmaBf16) {
    const __nv_bfloat16* Uh = reinterpret_cast<const __nv_bfloat16*>(Up);
    const __nv_bfloat16* Vh = reinterpret_cast<const __nv_bfloat16*>(Vp);
    const int mq = lane >> 3, r = lane & 7;
    uint32_t ah[MT][4], al[MT][4];
#pragma unroll
    for (int mi = 0; mi < MT; ++mi) {
      // matrices (i 0-7, k 0-7), (i 8-15, k 0-7), (i 0-7, k 8-15), (i 8-15, k 8-15)
      const int row = k0 + (mq >> 1) * 8 + r;
      const size_t off = (size_t)row * SU + (((2 * mi + (mq & 1)) ^ swz<ZU>(row)) << 3);
      ldsm_x4_t(ah[mi], Uh + off);
      ldsm_x4_t(al[mi], Uh + u_plane + off);
    }
#pragma unroll
    for (int nj = 0; nj < NTA; ++nj) {
      if (nj < jt0 || nj >= jt1) continue;
      // matrices (k 0-7, j), (k 8-15, j) from lanes 0-15
      const int row = k0 + (mq & 1) * 8 + r;
      const size_t off = (size_t)row * SV + ((nj ^ swz<ZV>(row)) << 3);
      uint32_t bh[2], bl[2];
      ldsm_x2_t(bh, Vh + off);
      ldsm_x2_t(bl, Vh + v_plane + off);
#pragma unroll
      for (int mi = 0; mi < MT; ++mi) {
        mma_bf16_16816(accx[mi][nj], al[mi], bh);
        mma_bf16_16816(acc[mi][nj], ah[mi], bh);
        mma_bf16_16816(accx[mi][nj], ah[mi], bl);
      }
    }
  } else {
    const float* U = reinterpret_cast<const float*>(Up);
    const float* V = reinterpret_cast<const float*>(Vp);
    const int g = lane >> 2, c = lane & 3;
    // rows k0 + c and k0 + c + 4 (k0 a multiple of 8): swizzle bits 0 and 1
    const int r0 = k0 + c, r1 = r0 + 4;
    auto at = [](int row, int col) { return (((col >> 2) ^ swz<ZU>(row)) << 2) + (col & 3); };
    auto bt = [](int row, int col) { return (((col >> 2) ^ swz<ZV>(row)) << 2) + (col & 3); };
    uint32_t ah[MT][4], al[MT][4];
#pragma unroll
    for (int mi = 0; mi < MT; ++mi) {
      const float* u0 = U + (size_t)r0 * SU;
      const float* u1 = U + (size_t)r1 * SU;
      split_tf32(u0[at(r0, 16 * mi + g)], ah[mi][0], al[mi][0]);
      split_tf32(u0[at(r0, 16 * mi + g + 8)], ah[mi][1], al[mi][1]);
      split_tf32(u1[at(r1, 16 * mi + g)], ah[mi][2], al[mi][2]);
      split_tf32(u1[at(r1, 16 * mi + g + 8)], ah[mi][3], al[mi][3]);
    }
#pragma unroll
    for (int nj = 0; nj < NTA; ++nj) {
      if (nj < jt0 || nj >= jt1) continue;
      uint32_t bh[2], bl[2];
      split_tf32(V[(size_t)r0 * SV + bt(r0, 8 * nj + g)], bh[0], bl[0]);
      split_tf32(V[(size_t)r1 * SV + bt(r1, 8 * nj + g)], bh[1], bl[1]);
#pragma unroll
      for (int mi = 0; mi < MT; ++mi) {
        mma_tf32_1688(accx[mi][nj], al[mi], bh);
        mma_tf32_1688(acc[mi][nj], ah[mi], bh);
        mma_tf32_1688(accx[mi][nj], ah[mi], bl);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------

template <int D, int P, int K>
__global__ void __launch_bounds__(kWarps * 32, MmaCfg<D, P, K>::MINB)
    row_mma_kernel(const DevMesh m, int mode, float* __restrict__ vals, float* __restrict__ rhs) {
  using Cfg = MmaCfg<D, P, K>;
  constexpr int N = Cfg::N, MT = Cfg::MT, NW = Cfg::NW, NT8 = Cfg::NT8, NTA = Cfg::NTA, NTV = Cfg::NTV;
  constexpr int C = Cfg::C, RW = Cfg::RW, SU = Cfg::SU, SV = Cfg::SV, G = Cfg::G, KS = Cfg::KS;
  constexpr int ZU = Cfg::ZU, ZV = Cfg::ZV;
  // separate accumulators for the cross products only where few tiles
  // would otherwise leave the MMA dependency chains exposed
  constexpr bool XACC = MT * NTA <= 2;
  constexpr int PT = Cfg::PT, PI = Cfg::PI, QT = Cfg::QT, SVL = sub_vals(D);
  constexpr int X = 4 * D;  // first scalar slot in PT
  constexpr size_t UPL = Cfg::u_plane, VPL = Cfg::v_plane;
  constexpr size_t UB = UPL * Cfg::ESZ * Cfg::NPL;  // bytes of the U planes
  constexpr size_t EU = (size_t)RW * SU * Cfg::ESZ, EV = (size_t)RW * SV * Cfg::ESZ;  // per element

  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* rule = reinterpret_cast<float*>(smem_raw);
  float* ctab = rule + QT * (D + 1);
  unsigned char* wb = smem_raw + Cfg::head_bytes + warp * Cfg::warp_bytes;
  unsigned char* Ust = wb;       // U planes: [plane][g][row][SU]
  unsigned char* Vst = wb + UB;  // V planes: [plane][g][row][SV]
  float* PTv = reinterpret_cast<float*>(wb + Cfg::stage_bytes);
  int* PIv = reinterpret_cast<int*>(wb + Cfg::stage_bytes + align_up(sizeof(float) * G * PT, 16));

  const float* vrule = m.rt.vol32 + (size_t)m.rt.vol_off[P] * (D + 1);
  for (int i = threadIdx.x; i < QT * (D + 1); i += blockDim.x) rule[i] = vrule[i];
  fill_ctab<D, float>(ctab, Cfg::NMAXC);
  __syncthreads();

  const float* SG = m.sg32;
  const float* HFR = m.hfr32;
  const float* FR = m.rt.face32;
  constexpr int FV = side_vals(D), RS = hf_rec_vals(D);
  const float* EG = m.eg32;

  const bool mat_vol = mode & kModeVol, mat_face = mode & kModeFace, do_rhs = mode & kModeRhs;
  const bool accum = mode & kModeAccum;
  const bool no_adv = m.pb.b[0] == 0.0 && m.pb.b[1] == 0.0 && m.pb.b[2] == 0.0 && m.pb.c == 0.0;
  const int base = m.elem_pstart[P], count = m.elem_pstart[P + 1] - base;
  const int ntiles = (count + G - 1) / G;
  constexpr int RT = N / 8;  // tile holding the load column
  const int gq = lane >> 2, cq = lane & 3;

  for (int tile = blockIdx.x * kWarps + warp; tile < ntiles; tile += gridDim.x * kWarps) {
    const int gcount = min(G, count - tile * G);
    __syncwarp();
    if (lane < G) {
      int* pi = PIv + lane * PI;
      float* pt = PTv + lane * PT;
      if (lane < gcount) {
        const int e = m.elem_perm[base + tile * G + lane];
        const int lrn = m.lq_ok && m.lq_ok[e] ? 1 : 0;
        pi[kPiElem] = e;
        pi[kPiLrn] = lrn;
        pi[kPiNvol] = lrn ? 28 : (m.eptr[e + 1] - m.eptr[e]) * QT;
        pi[kPiNface] = m.e_nqf[e];
        pi[kPiSub0] = m.eptr[e];
        pi[kPiHf0] = m.hf_ptr[e];
        pi[kPiNhf] = m.hf_ptr[e + 1] - m.hf_ptr[e];
        pi[kPiRow0] = m.row_ptr[e];
        pi[kPiNslot] = m.row_ptr[e + 1] - m.row_ptr[e] - 1;
        pi[kPiDpos] = m.diag_blk[e] - m.row_ptr[e];
        ElemPar<D, float> q;
        load_elem_par<D, float>(m, e, q);
#pragma unroll
        for (int d = 0; d < D; ++d) {
          pt[d] = q.ap[d];
          pt[D + d] = q.bp[d];
          pt[2 * D + d] = q.lo[d];
          pt[3 * D + d] = q.L[d];
        }
        pt[X + kPtC] = q.c;
        pt[X + kPtA] = q.a;
        pt[X + kPtR] = q.R;
      } else {
        pi[kPiElem] = -1;
        pi[kPiNvol] = 0;
        pi[kPiNface] = 0;
        pi[kPiNslot] = 0;
      }
    }
    __syncwarp();
    int nv_l = 0, nf_l = 0, ns_l = 0;
    if (lane < gcount) {
      nv_l = (PIv[lane * PI + kPiNvol] + C - 1) / C;
      nf_l = (PIv[lane * PI + kPiNface] + C - 1) / C;
      ns_l = PIv[lane * PI + kPiNslot];
    }
    const int nvch = __reduce_max_sync(0xffffffffu, nv_l);
    const int nfch = __reduce_max_sync(0xffffffffu, nf_l);
    const int nslot = __reduce_max_sync(0xffffffffu, ns_l);

    // acc / accx: the MMA accumulators of one chunk (at most RW / KS
    // k-steps); acct: the running sums, added in IEEE FP32 after every chunk,
    // so no accumulation chain inside the tensor cores spans more than one
    // chunk however many points an element has
    float acc[G][MT][NTA][4], accx[G][MT][NTA][4], acct[G][MT][NTA][4];
    auto flush = [&]() {
#pragma unroll
      for (int g = 0; g < G; ++g)
#pragma unroll
        for (int mi = 0; mi < MT; ++mi)
#pragma unroll
          for (int nj = 0; nj < NTA; ++nj)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              acct[g][mi][nj][r] += acc[g][mi][nj][r] + accx[g][mi][nj][r];
              acc[g][mi][nj][r] = accx[g][mi][nj][r] = 0.f;
            }
    };
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
      for (int mi = 0; mi < MT; ++mi)
#pragma unroll
        for (int nj = 0; nj < NTA; ++nj)
#pragma unroll
          for (int r = 0; r < 4; ++r) acc[g][mi][nj][r] = accx[g][mi][nj][r] = acct[g][mi][nj][r] = 0.f;

    // ---- volume points
    if (mat_vol || do_rhs) {
      for (int ch = 0; ch < nvch; ++ch) {
        if (lane < G * C) {
          const int g = lane / C, c = lane - (lane / C) * C, qv = ch * C + c;
          unsigned char* Ug = Ust + g * EU;
          unsigned char* Vg = Vst + g * EV;
          if (g < gcount && qv < PIv[g * PI + kPiNvol]) {
            const float* pt = PTv + g * PT;
            float xi[D], W;
            if (D == 2 && PIv[g * PI + kPiLrn]) {
              const float* LQ = m.lq32 + (size_t)PIv[g * PI + kPiElem] * 84;
              xi[0] = LQ[qv];
              xi[1 % D] = LQ[28 + qv];
              W = LQ[56 + qv];
            } else {
              const int t = qv / QT, r = qv - t * QT;
              const int sub = PIv[g * PI + kPiSub0] + t;
              float sv[SVL];
#pragma unroll
              for (int k = 0; k < SVL; ++k) sv[k] = SG[(size_t)k * m.nsub + sub];
              const float* rr = rule + r * (D + 1);
#pragma unroll
              for (int d = 0; d < D; ++d) {
                float v = sv[d] + rr[0] * sv[D + d] + rr[1] * sv[2 * D + d];
                if constexpr (D == 3) v += rr[2] * sv[3 * D + d];
                xi[d] = v;
              }
              W = rr[D] * sv[SVL - 1];
            }
            float Phi[N], Dd[D][N], Vv[N];
            basis_eval<D, P, float>(xi, Phi, Dd);
#pragma unroll
            for (int i = 0; i < N; ++i) {
              float adv = pt[X + kPtC] * Phi[i];
#pragma unroll
              for (int d = 0; d < D; ++d) adv += pt[D + d] * Dd[d][i];
              Vv[i] = W * adv;
            }
            float R0 = 0.f;
            if (do_rhs) {
              float x[D];
#pragma unroll
              for (int d = 0; d < D; ++d) x[d] = pt[2 * D + d] + (xi[d] + 1.f) * 0.5f * pt[3 * D + d];
              R0 = W * source_f<D, float>(m.pb, pt[X + kPtA], x);
            }
            put_row<K, SU, ZU, 16 * MT, N>(Ug, UPL, c, Phi, 0.f);
            put_row<K, SV, ZV, NW, N>(Vg, VPL, c, Vv, R0);
#pragma unroll
            for (int d = 0; d < D; ++d) {
              const float s = W * pt[d];
#pragma unroll
              for (int i = 0; i < N; ++i) Vv[i] = s * Dd[d][i];
              put_row<K, SU, ZU, 16 * MT, N>(Ug, UPL, (1 + d) * C + c, Dd[d], 0.f);
              put_row<K, SV, ZV, NW, N>(Vg, VPL, (1 + d) * C + c, Vv, 0.f);
            }
          } else {
#pragma unroll
            for (int t = 0; t < NTV; ++t) {
              zero_row<K, SU, 16 * MT>(Ug, UPL, t * C + c);
              zero_row<K, SV, NW>(Vg, VPL, t * C + c);
            }
          }
        }
        __syncwarp();
        bool gv[G];
#pragma unroll
        for (int g = 0; g < G; ++g) gv[g] = g < gcount && ch * C < PIv[g * PI + kPiNvol];
#pragma unroll 1
        for (int k0 = 0; k0 < RW; k0 += KS) {
          const int t = k0 / C;
          int jt0 = 0, jt1 = 0;
          if (mat_vol && !(t == 0 && no_adv)) {
            jt1 = NT8;
          } else if (do_rhs && t == 0) {
            jt0 = RT;
            jt1 = RT + 1;
          }
          if (jt1 <= jt0) continue;
#pragma unroll
          for (int g = 0; g < G; ++g)
            if (gv[g])
              mma_kstep<K, MT, NTA, SU, SV, ZU, ZV>(Ust + g * EU, UPL, Vst + g * EV, VPL, k0, jt0, jt1, acc[g],
                                                    XACC ? accx[g] : acc[g]);
        }
        flush();
        __syncwarp();
      }
    }

    // ---- own-face points
    if (mat_face || do_rhs) {
      for (int ch = 0; ch < nfch; ++ch) {
        if (lane < G * C) {
          const int g = lane / C, c = lane - (lane / C) * C, qv = ch * C + c;
          unsigned char* Ug = Ust + g * EU;
          unsigned char* Vg = Vst + g * EV;
          if (g < gcount && qv < PIv[g * PI + kPiNface]) {
            const float* pt = PTv + g * PT;
            int lo_ = PIv[g * PI + kPiHf0], hi_ = lo_ + PIv[g * PI + kPiNhf] - 1;
            while (lo_ < hi_) {
              const int mid = (lo_ + hi_ + 1) >> 1;
              if (m.hf_qoff[mid] <= qv)
                lo_ = mid;
              else
                hi_ = mid - 1;
            }
            const int hf = lo_;
            // the half face's record: own side, then J, sigma, b.n, nq (signed)
            const float* rec = HFR + (size_t)hf * RS;
            float sc[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) sc[j] = rec[2 * FV + j];
            const bool bnd = sc[3] < 0.f;
            const int nq = (int)(bnd ? -sc[3] : sc[3]);
            const int lq = qv - m.hf_qoff[hf];
            const float* fr = FR + (size_t)(m.rt.face_off[nq] + lq) * (D == 2 ? 2 : 3);
            float xi[D], np[D];
            hf_point<D, float>(rec, fr, xi, np);
            const float W = fr[D == 2 ? 1 : 2] * sc[0];
            const bool neu = sc[1] < 0.f;  // Neumann face: no matrix term, g_N in the load
            const float sig = neu ? 0.f : sc[1];
            const float bn = sc[2];
            const float kap = neu ? 0.f : bnd ? 1.f : 0.5f;
            const float a = pt[X + kPtA];
            const float upw = bn < 0.f ? bn : 0.f;
            float Phi[N], Dd[D][N], dn[N], V0[N], V1[N];
            basis_eval<D, P, float>(xi, Phi, Dd);
#pragma unroll
            for (int i = 0; i < N; ++i) {
              float v = 0.f;
#pragma unroll
              for (int d = 0; d < D; ++d) v += np[d] * Dd[d][i];
              dn[i] = v;
              V0[i] = W * (-kap * a * v + (sig - upw) * Phi[i]);
              V1[i] = W * (-kap * a * Phi[i]);
            }
            float R0 = 0.f, R1 = 0.f;
            if (do_rhs && bnd) {
              float x[D], gu[3], lap;
#pragma unroll
              for (int d = 0; d < D; ++d) x[d] = pt[2 * D + d] + (xi[d] + 1.f) * 0.5f * pt[3 * D + d];
              const float gd = exact_u<D, float>(m.pb, x, gu, &lap);
              R0 = W * (sig - upw) * gd;
              R1 = -W * a * gd;
              if (neu) {
                // g_N = a grad u . n_k, n_k = n' L / 2
                float gn = 0.f;
#pragma unroll
                for (int d = 0; d < D; ++d) gn += gu[d] * np[d] * pt[3 * D + d];
                R0 = W * 0.5f * a * gn;
                R1 = 0.f;
              }
            }
            put_row<K, SU, ZU, 16 * MT, N>(Ug, UPL, c, Phi, 0.f);
            put_row<K, SU, ZU, 16 * MT, N>(Ug, UPL, C + c, dn, 0.f);
            put_row<K, SV, ZV, NW, N>(Vg, VPL, c, V0, R0);
            put_row<K, SV, ZV, NW, N>(Vg, VPL, C + c, V1, R1);
          } else {
#pragma unroll
            for (int t = 0; t < 2; ++t) {
              zero_row<K, SU, 16 * MT>(Ug, UPL, t * C + c);
              zero_row<K, SV, NW>(Vg, VPL, t * C + c);
            }
          }
        }
        __syncwarp();
        bool gv[G];
#pragma unroll
        for (int g = 0; g < G; ++g) gv[g] = g < gcount && ch * C < PIv[g * PI + kPiNface];
        const int jt0 = mat_face ? 0 : RT, jt1 = mat_face ? NT8 : RT + 1;
#pragma unroll 1
        for (int k0 = 0; k0 < 2 * C; k0 += KS)
#pragma unroll
          for (int g = 0; g < G; ++g)
            if (gv[g])
              mma_kstep<K, MT, NTA, SU, SV, ZU, ZV>(Ust + g * EU, UPL, Vst + g * EV, VPL, k0, jt0, jt1, acc[g],
                                                    XACC ? accx[g] : acc[g]);
        flush();
        __syncwarp();
      }
    }

    // ---- write the diagonal blocks and the load vectors
#pragma unroll
    for (int g = 0; g < G; ++g) {
      if (g >= gcount) continue;
      const int e = PIv[g * PI + kPiElem];
      if (((mat_vol || mat_face) && !dg_in_range(m.status, m.blk_off[m.diag_blk[e]], (int64_t)N * N, m.nvals)) ||
          (do_rhs && !dg_in_range(m.status, m.dof_off[e], N, m.ndofs)))
        continue;
      const float Re = PTv[g * PT + X + kPtR];
      const float RR = Re * Re;
      float* out = vals + ((mat_vol || mat_face) ? m.blk_off[m.diag_blk[e]] : 0);
      float* rout = rhs + (do_rhs ? m.dof_off[e] : 0);
#pragma unroll
      for (int mi = 0; mi < MT; ++mi)
#pragma unroll
        for (int nj = 0; nj < NT8; ++nj)
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int i = 16 * mi + gq + 8 * (r >> 1), j = 8 * nj + 2 * cq + (r & 1);
            if (i >= N) continue;
            if (j < N && (mat_vol || mat_face)) {
              const float v = RR * ctab[i] * ctab[j] * acct[g][mi][nj][r];
              out[i * N + j] = accum ? out[i * N + j] + v : v;
            } else if (j == N && do_rhs) {
              rout[i] = Re * ctab[i] * acct[g][mi][nj][r];
            }
          }
    }

    // ---- off-diagonal blocks: one per neighbour, NW columns per pass
    if (mat_face) {
      for (int sl = 0; sl < nslot; ++sl) {
        __syncwarp();
        if (lane < G) {
          int* pi = PIv + lane * PI;
          if (lane < gcount && sl < pi[kPiNslot]) {
            const int bk = pi[kPiRow0] + sl + (sl >= pi[kPiDpos] ? 1 : 0);
            const int4 br = m.blk_rec[bk];  // neighbour, first half face, faces, neighbour degree
            const int k = br.x, pk = br.w;
            const int nq = (P > pk ? P : pk) + 1;
            const int qf = D == 2 ? nq : nq * nq;
            pi[kPiSBlk] = bk;
            pi[kPiSSide] = nq;
            pi[kPiSPk] = pk;
            pi[kPiSNk] = nbasis(D, pk);
            pi[kPiSF0] = br.y;
            pi[kPiSQF] = qf;
            pi[kPiSNpts] = br.z * qf;
            PTv[lane * PT + X + kPtAk] = float(m.a[k]);
            PTv[lane * PT + X + kPtRk] = EG[(size_t)(3 * D) * m.ne + k];
          } else {
            pi[kPiSNk] = 0;
            pi[kPiSNpts] = 0;
          }
        }
        __syncwarp();
        int np_l = 0, pc_l = 0;
        if (lane < gcount) {
          np_l = (PIv[lane * PI + kPiSNpts] + C - 1) / C;
          pc_l = (PIv[lane * PI + kPiSNk] + NW - 1) / NW;
        }
        const int nch = __reduce_max_sync(0xffffffffu, np_l);
        const int npass = __reduce_max_sync(0xffffffffu, pc_l);

        for (int pass = 0; pass < npass; ++pass) {
          const int col0 = pass * NW;
#pragma unroll
          for (int g = 0; g < G; ++g)
#pragma unroll
            for (int mi = 0; mi < MT; ++mi)
#pragma unroll
              for (int nj = 0; nj < NTA; ++nj)
#pragma unroll
                for (int r = 0; r < 4; ++r) acc[g][mi][nj][r] = accx[g][mi][nj][r] = acct[g][mi][nj][r] = 0.f;
          for (int ch = 0; ch < nch; ++ch) {
            __syncwarp();
            if (lane < G * C) {
              const int g = lane / C, c = lane - (lane / C) * C, qv = ch * C + c;
              unsigned char* Ug = Ust + g * EU;
              unsigned char* Vg = Vst + g * EV;
              const int* pi = PIv + g * PI;
              zero_row<K, SV, NW>(Vg, VPL, c);
              zero_row<K, SV, NW>(Vg, VPL, C + c);
              if (g < gcount && qv < pi[kPiSNpts] && col0 < pi[kPiSNk]) {
                const int qf = pi[kPiSQF];
                const int fi = qv / qf, lq = qv - fi * qf;
                const int nq = pi[kPiSSide];
                // the half face's record: both sides, then J, sigma, b.n
                const float* rec = HFR + (size_t)(pi[kPiSF0] + fi) * RS;
                const float* fr = FR + (size_t)(m.rt.face_off[nq] + lq) * (D == 2 ? 2 : 3);
                float xe[D], xk[D], ne_[D], nk_[D];
                hf_point<D, float>(rec, fr, xe, ne_);
                hf_point<D, float>(rec + FV, fr, xk, nk_);
                const float W = fr[D == 2 ? 1 : 2] * rec[2 * FV];
                const float sig = rec[2 * FV + 1];
                const float bn = rec[2 * FV + 2];
                const float upw = bn < 0.f ? bn : 0.f;
                const float ae = PTv[g * PT + X + kPtA];
                const float ak = PTv[g * PT + X + kPtAk];
                {
                  float Phi[N], Dd[D][N], dn[N];
                  basis_eval<D, P, float>(xe, Phi, Dd);
#pragma unroll
                  for (int i = 0; i < N; ++i) {
                    float v = 0.f;
#pragma unroll
                    for (int d = 0; d < D; ++d) v += ne_[d] * Dd[d][i];
                    dn[i] = v;
                  }
                  put_row<K, SU, ZU, 16 * MT, N>(Ug, UPL, c, Phi, 0.f);
                  put_row<K, SU, ZU, 16 * MT, N>(Ug, UPL, C + c, dn, 0.f);
                }
                auto sink = [&](int j, float phik, const float* dk) {
                  const int jj = j - col0;
                  if (jj < 0 || jj >= NW) return;
                  float dnk = 0.f;
#pragma unroll
                  for (int d = 0; d < D; ++d) dnk += nk_[d] * dk[d];
                  put_one<K, SV, ZV>(Vg, VPL, c, jj, W * (-0.5f * ak * dnk + (upw - sig) * phik));
                  put_one<K, SV, ZV>(Vg, VPL, C + c, jj, W * (0.5f * ae * phik));
                };
                nbr_basis<D, float>(pi[kPiSPk], xk, sink);
              } else {
                zero_row<K, SU, 16 * MT>(Ug, UPL, c);
                zero_row<K, SU, 16 * MT>(Ug, UPL, C + c);
              }
            }
            __syncwarp();
            bool gv[G];
            int gj[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
              const int* pi = PIv + g * PI;
              gv[g] = g < gcount && ch * C < pi[kPiSNpts] && col0 < pi[kPiSNk];
              gj[g] = gv[g] ? min(NTA, (pi[kPiSNk] - col0 + 7) / 8) : 0;
            }
#pragma unroll 1
            for (int k0 = 0; k0 < 2 * C; k0 += KS)
#pragma unroll
              for (int g = 0; g < G; ++g)
                if (gv[g])
                  mma_kstep<K, MT, NTA, SU, SV, ZU, ZV>(Ust + g * EU, UPL, Vst + g * EV, VPL, k0, 0, gj[g], acc[g],
                                                        XACC ? accx[g] : acc[g]);
            flush();
          }
          // this pass's columns of the off-diagonal blocks
#pragma unroll
          for (int g = 0; g < G; ++g) {
            if (g >= gcount) continue;
            const int* pi = PIv + g * PI;
            const int nk = pi[kPiSNk];
            if (col0 >= nk) continue;
            if (!dg_in_range(m.status, m.blk_off[pi[kPiSBlk]], (int64_t)N * nk, m.nvals)) continue;
            float* out = vals + m.blk_off[pi[kPiSBlk]];
            const float RR = PTv[g * PT + X + kPtR] * PTv[g * PT + X + kPtRk];
#pragma unroll
            for (int mi = 0; mi < MT; ++mi)
#pragma unroll
              for (int nj = 0; nj < NTA; ++nj)
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                  const int i = 16 * mi + gq + 8 * (r >> 1), j = col0 + 8 * nj + 2 * cq + (r & 1);
                  if (i < N && j < nk)
                    out[i * nk + j] = RR * ctab[i] * ctab[j] * acct[g][mi][nj][r];
                }
          }
        }
      }
    }
  }
}

template <int D, int P, int K>
inline int launch_row_mma_p(const DevMesh& m, int mode, float* vals, float* rhs, int sm_count, const LaunchOpts& lo,
                            Tracer* tr) {
  const int count = m.elem_pstart[P + 1] - m.elem_pstart[P];
  if (count <= 0) return 0;
  cudaStream_t st = lo.pst[P];
  if (tr && tr->on) {
    char name[48];
    snprintf(name, sizeof name, "row%dd_p%d_%s", D, P, K == kMmaBf16 ? "bf16x3" : "tf32x3");
    tr->begin(name, 0, P, 4, st);
  }
  if constexpr (P == 1) {
    // degree 1 (n = 3 or 4) is too small for 16-row tiles: the FP32 lane kernel
    auto k = row_lane_kernel<D, P, float, 2>;
    const int grid = resident_grid(k, 0, sm_count, lane_blocks<D, P, float>(count, 2), lo.occ_cap);
    k<<<grid, kWarps * 32, 0, st>>>(m, mode, vals, rhs);
  } else {
    using Cfg = MmaCfg<D, P, K>;
    static_assert(Cfg::total <= 227 * 1024, "tensor-core row kernel shared memory exceeds 227 KB");
    const int ntiles = (count + Cfg::G - 1) / Cfg::G;
    auto k = row_mma_kernel<D, P, K>;
    const int grid = resident_grid(k, Cfg::total, sm_count, (ntiles + kWarps - 1) / kWarps, lo.occ_cap);
    k<<<grid, kWarps * 32, Cfg::total, st>>>(m, mode, vals, rhs);
  }
  if (tr && tr->on) tr->end(st);
  return 1;
}

}  // namespace dg
