// k_tile.cu -- several element-Jacobi sweeps of a coarse P-level in one
// launch (Section 2.4, eq. smoothing_element_jacobi on the level system of
// Section 3), on tiles that carry their own halo.
//
// On the coarse levels one sweep is a short kernel whose time is mostly
// launch, ramp-up and drain.  Here each CTA owns a tile: a compact core of
// elements plus `depth` layers of face neighbours (host_tables.cpp
// build_tiles).  It loads the tile's states, factored blocks, scales, metrics,
// face geometry and FAS data into shared memory once, then runs n <= depth
// sweeps separated only by CTA barriers: sweep s (0-based) updates the
// elements up to halo layer n - 1 - s, whose neighbours all lie in the tile
// and were brought up to date by sweep s - 1.  The core ends with the values
// of n plain sweeps and is written back; halo elements are recomputed by the
// tiles that own them.  No grid-wide dependency is needed inside a launch.
//
// Per element and sweep the arithmetic is that of the one-sweep fused kernel
// in double-word arithmetic (fused_sweep_dw_kernel, k_fused.cu): the same
// operations in the same order, so the core's states are those of n fused
// sweeps bit for bit.  Gauge storage (p_ref != 0), mu = 0, no boundary faces.
#include "sweep_common.cuh"

namespace pmg {

template <int P, class W>
struct TileLayout {
  static constexpr int n1 = P + 1, N = n1 * n1, n = 4 * N, FP = 4 * n1;
  using Acc = typename Blk<W>::acc;
  // bytes per tile element, 8-byte arrays first
  static constexpr size_t per_elem = sizeof(double) * (2 * n        // rs, cs
                                                       + 2 * 4 * N  // state, ping-pong
                                                       + 5 * N      // metrics
                                                       + FP * 3     // face geometry
                                                       + 2 * 4 * N) // reference state, -S
                                     + sizeof(dw) * (2 * 4 * N + 16 * n1)   // Ft, Gt, jumps
                                     + sizeof(W) * n * n + sizeof(Acc) * n + sizeof(int) * 8;
  static size_t bytes(int M) { return (per_elem * (size_t)M + 127) / 128 * 128 + 256; }
};

template <int P, class W>
__global__ void __launch_bounds__(512, 1) tile_sweep_dw_kernel(
    const int* __restrict__ toff, const int* __restrict__ tlayer, const int* __restrict__ telems,
    const int* __restrict__ tlnbr, int depth, int nsweep, int E, const double* __restrict__ qin,
    double* __restrict__ qout, const double* __restrict__ met, const double* __restrict__ face,
    const int* __restrict__ nbr, OpTabW opw, OpTab op, PhysW k, double p_ref, double inv_odt,
    const double* __restrict__ S, const double* __restrict__ qref, const W* __restrict__ Dinv,
    const double* __restrict__ rs, const double* __restrict__ cs) {
  using L = TileLayout<P, W>;
  constexpr int n1 = L::n1, N = L::N, n = L::n, FP = L::FP;
  using Acc = typename L::Acc;
  const int tile = blockIdx.x;
  const int t0 = toff[tile], M = toff[tile + 1] - t0;
  const int* lay = tlayer + tile * (depth + 1);
  extern __shared__ __align__(128) unsigned char dsm[];
  // carve the tile arrays (M elements each)
  double* srs = reinterpret_cast<double*>(dsm);
  double* scs = srs + (size_t)M * n;
  double* sq0 = scs + (size_t)M * n;                 // [2][M][4][N]
  double* smt = sq0 + (size_t)2 * M * 4 * N;         // [M][5][N]
  double* sfg = smt + (size_t)M * 5 * N;             // [M][FP][3]
  double* sqo = sfg + (size_t)M * FP * 3;            // [M][4][N]
  double* sSv = sqo + (size_t)M * 4 * N;             // [M][4][N]
  dw* sFt = reinterpret_cast<dw*>(sSv + (size_t)M * 4 * N);   // [M][4][N]
  dw* sGt = sFt + (size_t)M * 4 * N;
  dw* sJ = sGt + (size_t)M * 4 * N;                  // [M][4 faces][4 vars][n1]
  W* sDinv = reinterpret_cast<W*>(sJ + (size_t)M * 16 * n1);   // [M][n*n]
  Acc* sr = reinterpret_cast<Acc*>(sDinv + (size_t)M * n * n); // [M][n]
  int* slnb = reinterpret_cast<int*>(sr + (size_t)M * n);      // [M][4]
  int* sfn = slnb + (size_t)M * 4;                   // [M][4]: neighbour face | reversed << 3
  __shared__ dw sD[n1][n1], sgL[n1], sgR[n1], swm[n1], swp[n1];
  __shared__ double slm[n1], slp[n1];
  const size_t plane = (size_t)E * N;

  // ---- load the tile
  for (int i = threadIdx.x; i < M * n * n; i += blockDim.x) {
    const int s = i / (n * n), r = i - s * (n * n);
    sDinv[i] = Dinv[(size_t)telems[t0 + s] * n * n + r];
  }
  for (int i = threadIdx.x; i < M * n; i += blockDim.x) {
    const int s = i / n, r = i - s * n;
    const int e = telems[t0 + s];
    srs[i] = rs[(size_t)e * n + r];
    scs[i] = cs[(size_t)e * n + r];
  }
  for (int i = threadIdx.x; i < M * 4; i += blockDim.x) {
    const int s = i >> 2, f = i & 3;
    const int e = telems[t0 + s];
    slnb[i] = tlnbr[(size_t)(t0 + s) * 4 + f];
    sfn[i] = nbr[(e * 4 + f) * 3 + 1] | (nbr[(e * 4 + f) * 3 + 2] << 3);
  }
  const int slot = threadIdx.x / FP, tf = threadIdx.x - slot * FP;
  const bool mine = slot < M;
  const bool own = mine && tf < N;
  const int f = tf / n1, kf = tf - f * n1;
  if (mine) {
    const int e = telems[t0 + slot];
    const double* g = face + (((size_t)e * 4 + f) * n1 + kf) * 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) sfg[((size_t)slot * FP + tf) * 3 + c] = __ldg(g + c);
    if (own) {
      const size_t gi = (size_t)e * N + tf;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        sq0[((size_t)slot * 4 + v) * N + tf] = __ldg(qin + v * plane + gi);
        sqo[((size_t)slot * 4 + v) * N + tf] = qref ? __ldg(qref + v * plane + gi) : 0.0;
        sSv[((size_t)slot * 4 + v) * N + tf] = S ? -__ldg(S + v * plane + gi) : 0.0;
      }
#pragma unroll
      for (int c = 0; c < 5; ++c) smt[((size_t)slot * 5 + c) * N + tf] = __ldg(met + c * plane + gi);
    }
  }
  if (threadIdx.x < n1 * n1) sD[threadIdx.x / n1][threadIdx.x % n1] = opw.D[threadIdx.x / n1][threadIdx.x % n1];
  if (threadIdx.x < n1) {
    sgL[threadIdx.x] = opw.gL[threadIdx.x];
    sgR[threadIdx.x] = opw.gR[threadIdx.x];
    swm[threadIdx.x] = opw.lm[threadIdx.x];
    swp[threadIdx.x] = opw.lp[threadIdx.x];
    slm[threadIdx.x] = op.lm[threadIdx.x];
    slp[threadIdx.x] = op.lp[threadIdx.x];
  }
  __syncthreads();

  for (int s = 0; s < nsweep; ++s) {
    const double* sqA = sq0 + (size_t)(s & 1) * M * 4 * N;
    double* sqB = sq0 + (size_t)((s + 1) & 1) * M * 4 * N;
    const bool act = mine && slot < lay[nsweep - 1 - s];
    const bool ow = act && tf < N;
    // phase 1: contravariant fluxes of the own point
    dw Q[4], rho = {0.0f, 0.0f};
    if (ow) {
#pragma unroll
      for (int v = 0; v < 4; ++v) Q[v] = dw_from_double(sqA[((size_t)slot * 4 + v) * N + tf]);
      rho = (Q[0] + k.p_ref) * rcp(Q[3]);
      const double* mt = smt + (size_t)slot * 5 * N;
      const dw a = dw_from_double(mt[0 * N + tf]), b = dw_from_double(mt[1 * N + tf]);
      const dw c = dw_from_double(mt[2 * N + tf]), d = dw_from_double(mt[3 * N + tf]);
      const dw H = k.Cp * Q[3] + half(Q[1] * Q[1] + Q[2] * Q[2]);
      const dw mx = rho * Q[1], my = rho * Q[2];
      const dw fx[4] = {mx, mx * Q[1] + Q[0], mx * Q[2], mx * H};
      const dw gy4[4] = {my, my * Q[1], my * Q[2] + Q[0], my * H};
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        dw_acc x, y;
        x.add_prod(a, fx[v]);
        x.add_prod(b, gy4[v]);
        y.add_prod(c, fx[v]);
        y.add_prod(d, gy4[v]);
        sFt[((size_t)slot * 4 + v) * N + tf] = x.value();
        sGt[((size_t)slot * 4 + v) * N + tf] = y.value();
      }
    }
    __syncthreads();
    // phase 2: face point (f, kf), the neighbour from the tile
    if (act) {
      const bool plus = (f == 1 || f == 2), eta = (f == 0 || f == 2), xi = !eta;
      const double* sqe = sqA + (size_t)slot * 4 * N;
      const double ref[4] = {sqe[0], 0.0, 0.0, sqe[3 * N]};
      const int ln = slnb[slot * 4 + f], fnr = sfn[slot * 4 + f];
      const int fn = fnr & 7, kn = (fnr >> 3) ? P - kf : kf;
      const bool etan = (fn == 0 || fn == 2), pn = (fn == 1 || fn == 2);
      const double* sqn = sqA + (size_t)ln * 4 * N;
      double sm[4], sp[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        double a = 0.0, b = 0.0;
#pragma unroll
        for (int m = 0; m < n1; ++m) {
          a = fma(plus ? slp[m] : slm[m], sqe[v * N + (eta ? m * n1 + kf : kf * n1 + m)] - ref[v], a);
          b = fma(pn ? slp[m] : slm[m], sqn[v * N + (etan ? m * n1 + kn : kn * n1 + m)] - ref[v], b);
        }
        sm[v] = a;
        sp[v] = b;
      }
      double qm[4], qp[4], dq[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        qm[v] = ref[v] + sm[v];
        qp[v] = ref[v] + sp[v];
        dq[v] = sp[v] - sm[v];
      }
      const double pgm = qm[0], pgp = qp[0];
      qm[0] += p_ref;
      qp[0] += p_ref;
      const double* g = sfg + ((size_t)slot * FP + tf) * 3;
      dw out[4];
      face_roe_dw(qm, qp, dq, pgm, pgp, g[0], g[1], g[2], k, out);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        dw_acc loc;
#pragma unroll
        for (int m = 0; m < n1; ++m)
          loc.add_prod(plus ? swp[m] : swm[m], xi ? sFt[((size_t)slot * 4 + v) * N + kf * n1 + m]
                                                  : sGt[((size_t)slot * 4 + v) * N + m * n1 + kf]);
        sJ[(((size_t)slot * 4 + f) * 4 + v) * n1 + kf] = (plus ? out[v] : -out[v]) - loc.value();
      }
    }
    __syncthreads();
    // phase 3: divergence, DG correction and level-system epilogue
    if (ow) {
      const int i = tf % n1, j = tf / n1;
      dw qc[4];
      if (qref) {
        dw Qo[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) Qo[v] = dw_from_double(sqo[((size_t)slot * 4 + v) * N + tf]);
        const dw rhoo = (Qo[0] + k.p_ref) * rcp(Qo[3]);
        qc[0] = rho - rhoo;
        qc[1] = rho * Q[1] - rhoo * Qo[1];
        qc[2] = rho * Q[2] - rhoo * Qo[2];
        qc[3] = (Q[0] - Qo[0]) * k.inv_gm1 +
                half(rho * (Q[1] * Q[1] + Q[2] * Q[2]) - rhoo * (Qo[1] * Qo[1] + Qo[2] * Qo[2]));
      } else {
        qc[0] = rho;
        qc[1] = rho * Q[1];
        qc[2] = rho * Q[2];
        qc[3] = rho * (Q[3] * k.inv_gm1 + half(Q[1] * Q[1] + Q[2] * Q[2]));
      }
      const dw invJ = dw_from_double(smt[((size_t)slot * 5 + 4) * N + tf]);
      const dw nodt = dw_from_double(-inv_odt);
      const dw* J4 = sJ + (size_t)slot * 16 * n1;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const dw* Ft = sFt + ((size_t)slot * 4 + v) * N;
        const dw* Gt = sGt + ((size_t)slot * 4 + v) * N;
        dw_acc acc;
#pragma unroll
        for (int m = 0; m < n1; ++m) {
          acc.add_prod(sD[i][m], Ft[j * n1 + m]);
          acc.add_prod(sD[j][m], Gt[m * n1 + i]);
        }
        acc.add_prod(sgL[i], J4[(3 * 4 + v) * n1 + j]);
        acc.add_prod(sgR[i], J4[(1 * 4 + v) * n1 + j]);
        acc.add_prod(sgL[j], J4[(0 * 4 + v) * n1 + i]);
        acc.add_prod(sgR[j], J4[(2 * 4 + v) * n1 + i]);
        dw_acc F;
        F.add_prod(-acc.value(), invJ);
        F.add_prod(qc[v], nodt);
        F.add(dw_from_double(sSv[((size_t)slot * 4 + v) * N + tf]));
        const int row = v * N + tf;
        sr[(size_t)slot * n + row] = scaled_in_dw<W>(F.value(), srs[(size_t)slot * n + row]);
      }
    }
    __syncthreads();
    // phase 4: block apply, rows 4 tf .. 4 tf + 3, into the other state buffer
    if (ow) {
      Acc acc[4] = {0, 0, 0, 0};
      const W* Dm = sDinv + (size_t)slot * n * n + 4 * tf;
#pragma unroll 4
      for (int kk = 0; kk < n; ++kk) {
        const Acc rk = sr[(size_t)slot * n + kk];
#pragma unroll
        for (int mm = 0; mm < 4; ++mm) acc[mm] = fma(blk_val(Dm[(size_t)kk * n + mm]), rk, acc[mm]);
      }
#pragma unroll
      for (int mm = 0; mm < 4; ++mm) {
        const int row = 4 * tf + mm;
        const int v = row / N, pt = row - v * N;
        const double xv = scaled_out<W>(acc[mm], scs[(size_t)slot * n + row]);
        sqB[((size_t)slot * 4 + v) * N + pt] = sqA[((size_t)slot * 4 + v) * N + pt] + xv;
      }
    }
    __syncthreads();
  }
  // write the core back
  const double* sqF = sq0 + (size_t)(nsweep & 1) * M * 4 * N;
  if (own && slot < lay[0]) {
    const int e = telems[t0 + slot];
#pragma unroll
    for (int v = 0; v < 4; ++v) qout[v * plane + (size_t)e * N + tf] = sqF[((size_t)slot * 4 + v) * N + tf];
  }
}

template <int P, class W>
static void tile_launch(const Ctx& c, const LevelDev& L, const double* qin, double* qout, int nsweep,
                        double inv_odt, const double* S, const double* qref, cudaStream_t s) {
  using Lay = TileLayout<P, W>;
  const int threads = (L.tile_M * Lay::FP + 31) / 32 * 32;
  tile_sweep_dw_kernel<P, W><<<L.n_tiles, threads, Lay::bytes(L.tile_M), s>>>(
      L.d_toff, L.d_tlayer, L.d_telems, L.d_tlnbr, L.tile_depth, nsweep, c.E, qin, qout, L.met, L.face,
      c.d_faces + 5 * c.n_faces, L.opw, L.op, c.phw, c.ph.p_ref, inv_odt, S, qref, (const W*)L.Dinv, L.rs, L.cs);
}

// One launch of nsweep (<= the tile depth) sweeps of a tiled level.
void launch_tile_sweeps(const Ctx& c, const LevelDev& L, const double* qin, double* qout, int nsweep,
                        double inv_odt, const double* S, const double* qref, int prec, cudaStream_t s) {
#define PMG_TL(PP)                                                                               \
  do {                                                                                           \
    if (prec == PMG_PREC_FP64) tile_launch<PP, double>(c, L, qin, qout, nsweep, inv_odt, S, qref, s); \
    else if (prec == PMG_PREC_BF16R)                                                             \
      tile_launch<PP, __nv_bfloat16>(c, L, qin, qout, nsweep, inv_odt, S, qref, s);              \
    else tile_launch<PP, float>(c, L, qin, qout, nsweep, inv_odt, S, qref, s);                   \
  } while (0)
  if (L.P == 0) PMG_TL(0);
  else PMG_TL(1);
#undef PMG_TL
}

// Shared memory a tile of M elements needs, or 0 if the level cannot be tiled.
size_t tile_smem_bytes(int P, int prec, int M) {
  if (P == 0)
    return prec == PMG_PREC_FP64 ? TileLayout<0, double>::bytes(M)
           : prec == PMG_PREC_BF16R ? TileLayout<0, __nv_bfloat16>::bytes(M) : TileLayout<0, float>::bytes(M);
  if (P == 1)
    return prec == PMG_PREC_FP64 ? TileLayout<1, double>::bytes(M)
           : prec == PMG_PREC_BF16R ? TileLayout<1, __nv_bfloat16>::bytes(M) : TileLayout<1, float>::bytes(M);
  return 0;
}

int tile_face_points(int P) { return 4 * (P + 1); }

cudaError_t prepare_tile_kernel(int P, int prec, size_t bytes) {
#define PMG_TP(PP, WT) \
  return cudaFuncSetAttribute(tile_sweep_dw_kernel<PP, WT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)
  if (P == 0) {
    if (prec == PMG_PREC_FP64) PMG_TP(0, double);
    if (prec == PMG_PREC_BF16R) PMG_TP(0, __nv_bfloat16);
    PMG_TP(0, float);
  }
  if (prec == PMG_PREC_FP64) PMG_TP(1, double);
  if (prec == PMG_PREC_BF16R) PMG_TP(1, __nv_bfloat16);
  PMG_TP(1, float);
#undef PMG_TP
}

}  // namespace pmg
