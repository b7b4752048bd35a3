// Mixed-precision mimetic stage kernel with TMA tiles.
//
// With nx a multiple of 4 the stage input y_s (halo 2) and B0s (halo 1)
// arrive in shared memory as cp.async.bulk.tensor boxes of all three
// components (component-major planes).  A box must start on a 16-byte
// boundary, so it starts 4 columns left of the tile (2 of them unused) and
// is YW = TX + 8 floats wide.  B (and 1/det G) is formed on the tile + halo 1
// into a ring of (x, y, z, w) vectors, the current at the tile's own nodes;
// stage s writes k_s and, pointwise, the next stage input y_{s+1} (see
// stage_kernels.cuh for the pipeline and the compact current).
//
// The CTA has WARPS warps; each thread owns R output rows of a plane (tile
// rows ty, ty + WARPS, ...), so the tile is TX x (WARPS R) nodes.  More rows
// per thread shrink the halo share of the B work and give each thread
// independent stencils to overlap.
#pragma once

#include "stage_kernels.cuh"

namespace glemur {

template <int WARPS, int R>
struct TmaGeo {
  static constexpr int NTH = 32 * WARPS;               // threads per CTA
  static constexpr int TH = WARPS * R;                 // tile height (nodes)
  static constexpr int BHt = TH + 2, BPt = BW * BHt;   // B tile (halo 1)
  static constexpr int YHt = TH + 4;                   // stage-input box height
  static constexpr int YCSt = YW * YHt, YPLt = 3 * YCSt;
  static constexpr int YSTRt = (YPLt * 4 + 127) / 128 * 32;  // ring slot stride (floats)
  static constexpr int ZHt = TH + 2;                   // B0 box height
  static constexpr int ZCSt = YW * ZHt, ZPLt = 3 * ZCSt;
  static constexpr int ZSTRt = (ZPLt * 4 + 127) / 128 * 32;  // B0 slot stride (floats)
  static constexpr unsigned YBYTESt = YPLt * 4, ZBYTESt = ZPLt * 4;
  static constexpr int BPTt = (BPt + NTH - 1) / NTH;   // B points per thread
  static_assert((BRING * BPt * 16) % 128 == 0, "B0 boxes must stay 128-byte aligned");
  static constexpr size_t smem_bytes() {
    return 128 + (size_t)XRING * YSTRt * 4 + (size_t)BRING * BPt * 16 + (size_t)2 * ZSTRt * 4;
  }
};

// The B-tile points a thread computes and what does not change between
// planes: index in the stage-input box, in-plane node offset, the x/y
// stencil codes, ownership (energy sum) and boundary count (zeta).
template <class Gm>
struct TmaBPts {
  static constexpr int BPT = Gm::BPTt;
  int x0[BPT], nxy[BPT], code[BPT];
  __device__ __forceinline__ void init(int i0, int j0, int nx, int ny) {
#pragma unroll
    for (int t = 0; t < BPT; ++t) {
      const int p = threadIdx.x + t * Gm::NTH;
      x0[t] = -1;
      nxy[t] = 0;
      code[t] = 0;
      if (p >= Gm::BPt) continue;
      const int bx = p % BW, by = p / BW;
      const int gi = i0 - 1 + bx, gj = j0 - 1 + by;
      if (gi < 0 || gi >= nx || gj < 0 || gj >= ny) continue;
      x0[t] = (by + 1) * YW + bx + 3;
      nxy[t] = gj * nx + gi;
      const int sx = gi == 0 ? 1 : (gi == nx - 1 ? 2 : 0);
      const int sy = gj == 0 ? 1 : (gj == ny - 1 ? 2 : 0);
      const int own = bx >= 1 && bx <= TX && by >= 1 && by <= Gm::TH;
      code[t] = sx | (sy << 2) | (own << 4) | (((sx != 0) + (sy != 0)) << 5);
    }
  }
};

// o = a - b for points of (possibly different) component-major planes with
// component stride CS.
template <int CS>
__device__ __forceinline__ void tsub(const float* pa, int ia, const float* pb, int ib,
                                     float o[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) o[c] = pa[ia + c * CS] - pb[ib + c * CS];
}
// one-sided second-order difference sgn (4 p1 - 3 p0 - p2)
template <int CS>
__device__ __forceinline__ void tside(const float* p0, int i0, const float* p1, int i1,
                                      const float* p2, int i2, float sgn, float o[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c)
    o[c] = sgn * ((4.0f * p1[i1 + c * CS] - 3.0f * p0[i0 + c * CS]) - p2[i2 + c * CS]);
}

// Stage-input planes q-2 .. q+2 around plane q.
struct TmaRing {
  const float* ym2;
  const float* ym;
  const float* yq;
  const float* yp;
  const float* yp2;
};

// B (and 1/det G) at every node of plane q in the tile + halo 1, from the
// stage-input planes around q, into the B plane `bq`; B0s from the B0 box
// `zp` or, if null, from the registers `b0v` (x0 - YW indexes the B0 box).
template <class Gm>
__device__ __forceinline__ void tma_compute_B(const StageArgs<float>& a, int q, int k0, int k1,
                                              const TmaBPts<Gm>& bp,
                                              const float* __restrict__ zp,
                                              const float (*b0v)[3], const TmaRing& Rg,
                                              V4<float>* __restrict__ bq, bool diag,
                                              Acc<float>& acc) {
  constexpr int CS = Gm::YCSt, ZC = Gm::ZCSt;
  const float h20 = a.h2f[0], h21 = a.h2f[1], h22 = a.h2f[2];
  const int sz = q == 0 ? 1 : (q == a.nz - 1 ? 2 : 0);
  const bool own_plane = diag && q >= k0 && q < k1;
#pragma unroll
  for (int t = 0; t < TmaBPts<Gm>::BPT; ++t) {
    const int x0 = bp.x0[t];
    if (x0 < 0) continue;
    const int p = threadIdx.x + t * Gm::NTH;
    const int code = bp.code[t];
    const int sx = code & 3, sy = (code >> 2) & 3;
    const float* yq = Rg.yq;
    float g[3][3];
    if (sx == 0)
      tsub<CS>(yq, x0 + 1, yq, x0 - 1, g[0]);
    else if (sx == 1)
      tside<CS>(yq, x0, yq, x0 + 1, yq, x0 + 2, 1.0f, g[0]);
    else
      tside<CS>(yq, x0, yq, x0 - 1, yq, x0 - 2, -1.0f, g[0]);
    if (sy == 0)
      tsub<CS>(yq, x0 + YW, yq, x0 - YW, g[1]);
    else if (sy == 1)
      tside<CS>(yq, x0, yq, x0 + YW, yq, x0 + 2 * YW, 1.0f, g[1]);
    else
      tside<CS>(yq, x0, yq, x0 - YW, yq, x0 - 2 * YW, -1.0f, g[1]);
    if (sz == 0)
      tsub<CS>(Rg.yp, x0, Rg.ym, x0, g[2]);
    else if (sz == 1)
      tside<CS>(yq, x0, Rg.yp, x0, Rg.yp2, x0, 1.0f, g[2]);
    else
      tside<CS>(yq, x0, Rg.ym, x0, Rg.ym2, x0, -1.0f, g[2]);
    g[0][0] += h20;
    g[1][1] += h21;
    g[2][2] += h22;
    const float det = det3(g[0], g[1], g[2]);
    acc.bad |= det <= 0.0f;  // NaN: reported by the error norm
    const float r = recip(det);
    float b0, b1, b2;
    if (zp) {
      const int zi = x0 - YW;
      b0 = zp[zi];
      b1 = zp[zi + ZC];
      b2 = zp[zi + 2 * ZC];
    } else {
      b0 = b0v[t][0];
      b1 = b0v[t][1];
      b2 = b0v[t][2];
    }
    float B[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) B[c] = (g[0][c] * b0 + g[1][c] * b1 + g[2][c] * b2) * r;
    bq[p] = V4<float>{B[0], B[1], B[2], r};
    if (own_plane && (code & 16)) {
      const int nb = ((code >> 5) & 3) + (sz != 0);
      const float zeta = nb == 0 ? 1.0f : nb == 1 ? 0.5f : nb == 2 ? 0.25f : 0.125f;
      acc.add_e(zeta * dot3(B, B) * det);
    }
  }
}

// Mimetic current and velocity at the thread's node of tile row `row`
// (node index n) of a plane: stage-input planes ym, yq, yp and B planes bm,
// bq, bp around it.
template <class Gm, int S>
__device__ __forceinline__ void tma_mimetic_out(const StageArgs<float>& a, int row, int n,
                                                const float* __restrict__ ym,
                                                const float* __restrict__ yq,
                                                const float* __restrict__ yp,
                                                const V4<float>* __restrict__ bm,
                                                const V4<float>* __restrict__ bq,
                                                const V4<float>* __restrict__ bp,
                                                const Centre<float, float, S>& ce, float* dout,
                                                const float* an, const DevState* st, bool diag,
                                                Acc<float>& acc) {
  constexpr int CS = Gm::YCSt;
  const int tx = threadIdx.x % TX;
  const int x0 = (row + 2) * YW + (tx + 4);
  const int b0i = (row + 1) * BW + (tx + 1);
  float g0[3], g1[3], g2[3], P0[3], P1[3], P2[3];
  tsub<CS>(yq, x0 + 1, yq, x0 - 1, g0);
  tsub<CS>(yq, x0 + YW, yq, x0 - YW, g1);
  tsub<CS>(yp, x0, ym, x0, g2);
  vsub(bq[b0i + 1], bq[b0i - 1], P0);
  vsub(bq[b0i + BW], bq[b0i - BW], P1);
  vsub(bp[b0i], bm[b0i], P2);
  const V4<float> bc = bq[b0i];
  const float B[3] = {bc.x, bc.y, bc.z};
  g0[0] += a.h2f[0];
  g1[1] += a.h2f[1];
  g2[2] += a.h2f[2];
  const float c0 = dot3(P1, g2) - dot3(P2, g1);
  const float c1 = dot3(P2, g0) - dot3(P0, g2);
  const float c2 = dot3(P0, g1) - dot3(P1, g0);
  const float rdet = bc.w;
  float J[3], u[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) J[c] = (c0 * g0[c] + c1 * g1[c] + c2 * g2[c]) * rdet;
  u[0] = J[1] * B[2] - J[2] * B[1];
  u[1] = J[2] * B[0] - J[0] * B[2];
  u[2] = J[0] * B[1] - J[1] * B[0];
  emit_centre<float, float, S>(a, n, u, J, B, ce, dout, an, st, diag, acc);
}

// B0s at the thread's B points of plane q, from global memory (prologue).
template <class Gm>
__device__ __forceinline__ void tma_load_B0(const StageArgs<float>& a, int q,
                                            const TmaBPts<Gm>& bp, float (*out)[3]) {
  const int N = a.nx * a.ny * a.nz;
  const int nq = q * a.nx * a.ny;
#pragma unroll
  for (int t = 0; t < TmaBPts<Gm>::BPT; ++t) {
    if (bp.x0[t] < 0) continue;
    const int n = nq + bp.nxy[t];
#pragma unroll
    for (int c = 0; c < 3; ++c) out[t][c] = __ldg(&a.B0s[c * N + n]);
  }
}

// Stage S (0..5).  Iteration m: thread 0 arms barrier m & 1 and issues the
// boxes of y plane m+4 and B0 plane m+3; every thread waits for the boxes
// issued in iteration m-1 (y plane m+3, B0 plane m+2), forms B at plane m+2
// and the current at its R nodes of plane m.  The prologue's boxes complete
// on a third barrier.  Every wait is bounded: a wait that gives up raises
// FLAG_TIMEOUT, and thread 0 then waits (bounded again) for every box the
// CTA still has in flight -- those of the barrier that timed out and of the
// current iteration -- before the CTA returns.  After a real stall that
// second wait can give up too: it then only delays the exit.  The test
// hook (a.tma_test) adds a fourth barrier that no copy completes to the
// prologue wait (1) or to the first wait inside the loop (2); the real
// copies do complete, so the clean-up waits see them land.
template <int WARPS, int R, int S>
__device__ __forceinline__ void stage_mimetic_tma_body(const StageArgs<float>& a,
                                                       const TmaMaps& maps) {
  using Gm = TmaGeo<WARPS, R>;
  constexpr bool FINAL = S == 5;
  const DevState* st = a.st;
  if (st->flags & FLAG_TIMEOUT) return;  // an earlier stage of this attempt gave up
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double red[32];
  __shared__ uint64_t bars[4];
  unsigned char* base =
      smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);  // 128-byte aligned
  float* yr = reinterpret_cast<float*>(base);                          // [XRING][YSTRt]
  V4<float>* bs = reinterpret_cast<V4<float>*>(yr + XRING * Gm::YSTRt); // [BRING][BPt]
  float* zr = reinterpret_cast<float*>(bs + BRING * Gm::BPt);          // [2][ZSTRt]
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * Gm::TH;
  const int k0 = blockIdx.z * a.kz, k1 = min(a.nz, k0 + a.kz);
  const int N = a.nx * a.ny * a.nz, nxy = a.nx * a.ny;
  const int cur = st->cur;
  const float* d = a.d[cur];
  float* dout = const_cast<float*>(a.d[cur ^ 1]);
  const CUtensorMap* ymap = S == 0 ? &maps.d[cur] : &maps.ys[S & 1];
  float an[S < 5 ? S + 1 : 1];  // dt a_{S+1, j}: the next stage input
#pragma unroll
  for (int j = 0; j < (S < 5 ? S + 1 : 0); ++j) an[j] = coef_a<float>(st, S + 1, j);
  const bool diag = a.diag != 0;
  Acc<float> acc;
  TmaBPts<Gm> bp;
  bp.init(i0, j0, a.nx, a.ny);
  // the thread's output rows ty + r WARPS
  const int gi = i0 + threadIdx.x % TX, ty = threadIdx.x / TX;
  bool out_xy[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int gj = j0 + ty + r * WARPS;
    out_xy[r] = gi >= 1 && gi <= a.nx - 2 && gj >= 1 && gj <= a.ny - 2;
  }
  const int nxy_out = (j0 + ty) * a.nx + gi;
  if (threadIdx.x == 0) {
    for (int i = 0; i < 4; ++i) mbar_init(&bars[i], 1);
    fence_barrier_init();
    // test hook: a phase that waits for 16 bytes no copy delivers
    if (a.tma_test) mbar_arrive_expect_tx(&bars[3], 16u);
    // prologue boxes: input planes k0-2 .. k0+3, B0 of plane k0+2
    unsigned bytes = 0;
    for (int q = k0 - 2; q <= k0 + 3; ++q)
      if (q >= 0 && q < a.nz && q <= k1 + 1) bytes += Gm::YBYTESt;
    const bool z2 = k0 + 2 < a.nz && k0 + 2 <= k1;
    if (z2) bytes += Gm::ZBYTESt;
    mbar_arrive_expect_tx(&bars[2], bytes);
    for (int q = k0 - 2; q <= k0 + 3; ++q)
      if (q >= 0 && q < a.nz && q <= k1 + 1)
        tma_load_4d(yr + xslot(q) * Gm::YSTRt, ymap, i0 - 4, j0 - 2, q, 0, &bars[2]);
    if (z2)
      tma_load_4d(zr + ((k0 + 2) & 1) * Gm::ZSTRt, &maps.b0, i0 - 4, j0 - 1, k0 + 2, 0,
                  &bars[2]);
  }
  __syncthreads();
  {
    bool ok = mbar_wait_bounded(&bars[2], 0);
    if (a.tma_test == 1) ok = ok && mbar_wait_bounded(&bars[3], 0);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicOr(&a.st->flags, FLAG_TIMEOUT);
        mbar_wait_bounded(&bars[2], 0);  // the prologue's boxes still in flight
      }
      return;
    }
  }
  for (int q = k0 - 1; q <= k0 + 1; ++q)
    if (q >= 0 && q < a.nz && q <= k1) {
      float b0v[TmaBPts<Gm>::BPT][3];
      tma_load_B0<Gm>(a, q, bp, b0v);
      const TmaRing Rg{yr + xslot(q - 2) * Gm::YSTRt, yr + xslot(q - 1) * Gm::YSTRt,
                       yr + xslot(q) * Gm::YSTRt, yr + xslot(q + 1) * Gm::YSTRt,
                       yr + xslot(q + 2) * Gm::YSTRt};
      tma_compute_B<Gm>(a, q, k0, k1, bp, nullptr, b0v, Rg, bs + bslot(q) * Gm::BPt, diag, acc);
    }
  __syncthreads();
  // ring slot offsets of the y_s planes m-1 .. m+4 and the B planes
  // m-1 .. m+2; one plane on, each list rotates by one (the slot of plane
  // m-1 is the slot of plane m+5, resp. m+3)
  int yo[6], bo[4];
#pragma unroll
  for (int dd = 0; dd < 6; ++dd) yo[dd] = xslot(k0 + dd - 1) * Gm::YSTRt;
#pragma unroll
  for (int dd = 0; dd < 4; ++dd) bo[dd] = bslot(k0 + dd - 1) * Gm::BPt;
  // centre values (d, k_j) of the output nodes, loaded one plane ahead: the
  // loads for plane m+1 are issued before the barrier that ends plane m
  Centre<float, float, S> ce[R];
  {
    const bool zin0 = k0 >= 1 && k0 <= a.nz - 2;
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (zin0 && out_xy[r]) ce[r].issue(a, d, N, k0 * nxy + nxy_out + r * WARPS * a.nx);
  }
  for (int m = k0; m < k1; ++m) {
    const int it = m - k0;
    const float* yl[6];
#pragma unroll
    for (int dd = 0; dd < 6; ++dd) yl[dd] = yr + yo[dd];
    V4<float>* bl[4];
#pragma unroll
    for (int dd = 0; dd < 4; ++dd) bl[dd] = bs + bo[dd];
    if (threadIdx.x == 0) {
      const bool ly = m + 4 < a.nz && m + 4 <= k1 + 1;
      const bool lz = m + 3 < a.nz && m + 3 <= k1;
      uint64_t* bar = &bars[it & 1];
      mbar_arrive_expect_tx(bar, (ly ? Gm::YBYTESt : 0u) + (lz ? Gm::ZBYTESt : 0u));
      if (ly) tma_load_4d(const_cast<float*>(yl[5]), ymap, i0 - 4, j0 - 2, m + 4, 0, bar);
      if (lz)
        tma_load_4d(zr + ((m + 3) & 1) * Gm::ZSTRt, &maps.b0, i0 - 4, j0 - 1, m + 3, 0, bar);
    }
    const bool zin = m >= 1 && m <= a.nz - 2;
    if (it > 0) {
      const int pi = it - 1;
      bool ok = mbar_wait_bounded(&bars[pi & 1], (pi >> 1) & 1);
      if (a.tma_test == 2 && it == 1) ok = ok && mbar_wait_bounded(&bars[3], 0);
      if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
          atomicOr(&a.st->flags, FLAG_TIMEOUT);
          // let the boxes of the barrier that gave up and of this
          // iteration land before the CTA leaves
          mbar_wait_bounded(&bars[pi & 1], (pi >> 1) & 1);
          mbar_wait_bounded(&bars[it & 1], (it >> 1) & 1);
        }
        return;
      }
    }
    const int qb = m + 2;  // B plane computed in this iteration
    if (qb < a.nz && qb <= k1) {
      const TmaRing Rg{yl[1], yl[2], yl[3], yl[4], yl[5]};  // planes m .. m+4
      tma_compute_B<Gm>(a, qb, k0, k1, bp, zr + (qb & 1) * Gm::ZSTRt, nullptr, Rg, bl[3], diag,
                        acc);
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (zin && out_xy[r])
        tma_mimetic_out<Gm, S>(a, ty + r * WARPS, m * nxy + nxy_out + r * WARPS * a.nx, yl[0],
                               yl[1], yl[2], bl[0], bl[1], bl[2], ce[r], dout, an, st, diag,
                               acc);
    if (m + 1 < k1) {
      const bool zin1 = m + 1 >= 1 && m + 1 <= a.nz - 2;
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (zin1 && out_xy[r])
          ce[r].issue(a, d, N, (m + 1) * nxy + nxy_out + r * WARPS * a.nx);
    }
    const int y_first = yo[0], b_first = bo[0];
#pragma unroll
    for (int dd = 0; dd < 5; ++dd) yo[dd] = yo[dd + 1];
    yo[5] = y_first;
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) bo[dd] = bo[dd + 1];
    bo[3] = b_first;
    __syncthreads();
  }
  pdl_trigger();
  if (__syncthreads_or(acc.bad) && threadIdx.x == 0)
    atomicOr(&a.st->flags, S == 0 ? FLAG_COLLAPSED : FLAG_FOLDED_TRIAL);
  write_partials<float, float>(a, FINAL, diag, acc, red);
}

// The kernel: the body above (which may leave early on a timed-out wait).
template <int WARPS, int R, int S, int MINB>
__global__ void __launch_bounds__(32 * WARPS, MINB)
    k_stage_mimetic_tma(const StageArgs<float> a, const __grid_constant__ TmaMaps maps) {
  pdl_wait();
  const DevState* st = a.st;
  if (!a.force && (st->status != ST_OK || st->n_accept >= st->target)) return;
  stage_mimetic_tma_body<WARPS, R, S>(a, maps);
}

// Launch stage `stage` (0..5) of the TMA mimetic kernel on `grid`.
template <int WARPS, int R, int MINB>
cudaError_t launch_stage_tma_t(const StageArgs<float>& a, const TmaMaps& maps, int stage,
                               dim3 grid, cudaStream_t s) {
  using Gm = TmaGeo<WARPS, R>;
  const size_t smem = Gm::smem_bytes();
  const int nt = Gm::NTH;
  switch (stage) {
    case 0: return launch_pdl(k_stage_mimetic_tma<WARPS, R, 0, MINB>, grid, dim3(nt), smem, s, a, maps);
    case 1: return launch_pdl(k_stage_mimetic_tma<WARPS, R, 1, MINB>, grid, dim3(nt), smem, s, a, maps);
    case 2: return launch_pdl(k_stage_mimetic_tma<WARPS, R, 2, MINB>, grid, dim3(nt), smem, s, a, maps);
    case 3: return launch_pdl(k_stage_mimetic_tma<WARPS, R, 3, MINB>, grid, dim3(nt), smem, s, a, maps);
    case 4: return launch_pdl(k_stage_mimetic_tma<WARPS, R, 4, MINB>, grid, dim3(nt), smem, s, a, maps);
    case 5: return launch_pdl(k_stage_mimetic_tma<WARPS, R, 5, MINB>, grid, dim3(nt), smem, s, a, maps);
    default: return cudaErrorInvalidValue;
  }
}

template <int WARPS, int R, int MINB>
cudaError_t prepare_stage_tma_t() {
  const int sm = (int)TmaGeo<WARPS, R>::smem_bytes();
  const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_stage_mimetic_tma<WARPS, R, 0, MINB>, at, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_stage_mimetic_tma<WARPS, R, 1, MINB>, at, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_stage_mimetic_tma<WARPS, R, 2, MINB>, at, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_stage_mimetic_tma<WARPS, R, 3, MINB>, at, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_stage_mimetic_tma<WARPS, R, 4, MINB>, at, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_stage_mimetic_tma<WARPS, R, 5, MINB>, at, sm);
  return e;
}

template <int WARPS, int R, int MINB>
int stage_tma_ctas_per_sm_t() {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stage_mimetic_tma<WARPS, R, 3, MINB>,
                                                TmaGeo<WARPS, R>::NTH,
                                                TmaGeo<WARPS, R>::smem_bytes());
  return n;
}

}  // namespace glemur
