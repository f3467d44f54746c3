// net_kernels.cuh -- forward and backward kernels of the gauge-covariant
// preconditioner network (definition in include/stag.h, stag_net_create).
//
// Activations are full-lattice fields stored per parity: [2][Vh][C][3]
// complex FP32, the C channels of a site contiguous.  A layer reads, for each
// of its 9 directions d, the fat-link hop of the staggered operator (the
// library's FP32 link copy: entries mu*CPM + 0..17 of the output parity's
// chunk list hold the +mu and -mu hop matrices with eta and 1/2 folded in)
// and the neighbour's channels, transports them, and mixes channels with the
// layer's real weights (stored as bfloat16, held in shared memory as FP32,
// FP32 accumulation).
#pragma once
#include <cuda_bf16.h>

#include "dslash_impl.cuh"

namespace stag {

constexpr int NET_NDIR = 9;
constexpr int NET_MAXC = 16;

struct NetGeom {
  Geom g;
  const uint4* links[2];  // FP32 link chunks for output parity 0 and 1
  int cpm;                // complex entries per direction in the chunk list
};

__device__ __forceinline__ float2* act_ptr(float2* a, int C, int Vh, int p, int s) {
  return a + (((size_t)p * Vh + s) * C) * 3;
}
__device__ __forceinline__ const float2* act_ptr(const float2* a, int C, int Vh, int p, int s) {
  return a + (((size_t)p * Vh + s) * C) * 3;
}

// The 3x3 hop matrix of direction d (1..8) at site s of parity p.
__device__ __forceinline__ void load_hop_matrix(const NetGeom& ng, int p, int s, int d, float2 w[9]) {
  const int mu = (d - 1) >> 1;
  const int k0 = mu * ng.cpm + ((d & 1) ? 0 : 9);  // FP32: 2 complex per chunk
  const uint4* L = p ? ng.links[1] : ng.links[0];
  const int Vh = ng.g.Vh;
  // chunks c0 .. c0 + 4 hold entries 2 c0 .. 2 c0 + 9; the matrix starts at
  // the first entry (k0 even) or the second (k0 odd).  Indices into w stay
  // compile-time constants so that w lives in registers.
  const bool odd = k0 & 1;
  const uint4* src = L + (size_t)(k0 >> 1) * Vh + s;
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const uint4 c = __ldg(src + (size_t)j * Vh);
    const float2 a = make_float2(__uint_as_float(c.x), __uint_as_float(c.y));
    const float2 b = make_float2(__uint_as_float(c.z), __uint_as_float(c.w));
    if (j > 0) w[2 * j - 1] = odd ? a : w[2 * j - 1];
    if (j < 4) w[2 * j + 1] = odd ? w[2 * j + 1] : b;
    w[2 * j] = odd ? b : a;
  }
}

// Neighbour (parity, index) of (p, s) for direction d (0: itself).
__device__ __forceinline__ void net_neighbour(const NetGeom& ng, int p, int s, int d, int& np, int& ns) {
  if (d == 0) {
    np = p;
    ns = s;
    return;
  }
  const int mu = (d - 1) >> 1;
  Coord c = cb_coords(ng.g, s, p);
  ns = cb_neighbour(ng.g, s, c, mu, (d & 1) ? 1 : -1);
  np = 1 - p;
}

// pre_c(x) = sum_d sum_c' W[d][c][c'] (T_d h_c')(x); GATE: out = pre * sigmoid(|pre|^2 - b_c).
// Weights come in as bfloat16 [9][COUT][CIN]; wsign[d] multiplies direction d
// (used for the adjoint pass: T_{1+2mu}^dag = -T_{2+2mu}).
template <int CIN, int COUT, bool GATE>
__global__ void __launch_bounds__(128) k_net_layer(NetGeom ng, const float2* __restrict__ hin, float2* __restrict__ pre,
                                                  float2* __restrict__ hout, const __nv_bfloat16* __restrict__ W,
                                                  const float* __restrict__ bias, int transpose) {
  __shared__ float sw[NET_NDIR * COUT * CIN];
  for (int i = threadIdx.x; i < NET_NDIR * COUT * CIN; i += blockDim.x) {
    // transpose != 0: the adjoint layer -- W'[d][c][c'] = sign(d) * W[partner(d)][c'][c]
    if (!transpose) {
      sw[i] = __bfloat162float(W[i]);
    } else {
      const int d = i / (COUT * CIN), rem = i % (COUT * CIN), c = rem / CIN, cp = rem % CIN;
      const int dd = d == 0 ? 0 : ((d & 1) ? d + 1 : d - 1);
      const float sg = d == 0 ? 1.f : -1.f;
      sw[i] = sg * __bfloat162float(W[(dd * CIN + cp) * COUT + c]);  // source layer is [9][CIN][COUT]
    }
  }
  __syncthreads();
  const int Vh = ng.g.Vh;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = idx < 2 * Vh;
  const int p = valid ? idx / Vh : 0, s = valid ? idx - p * Vh : 0;
  float2 acc[COUT][3];
#pragma unroll
  for (int c = 0; c < COUT; ++c)
#pragma unroll
    for (int i = 0; i < 3; ++i) acc[c][i] = make_float2(0.f, 0.f);
#pragma unroll 1
  for (int d = 0; d < (valid ? NET_NDIR : 0); ++d) {
    int np, ns;
    net_neighbour(ng, p, s, d, np, ns);
    float2 w[9];
    if (d) load_hop_matrix(ng, p, s, d, w);
    const float2* src = act_ptr(hin, CIN, Vh, np, ns);
    if constexpr (COUT == 1 && CIN > 1) {
      // one output channel: mix first, then transport once (T_d is linear
      // and the weights are real, so sum_c' W T_d h_c' = T_d sum_c' W h_c')
      float2 m[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      const float* wr = sw + d * CIN;
#pragma unroll 4
      for (int cp = 0; cp < CIN; ++cp) {
        const float k = wr[cp];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const float2 v = __ldg(src + cp * 3 + i);
          m[i].x = fmaf(k, v.x, m[i].x);
          m[i].y = fmaf(k, v.y, m[i].y);
        }
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        if (d) {
#pragma unroll
          for (int j = 0; j < 3; ++j) cmac(acc[0][i], w[3 * i + j], m[j]);
        } else {
          acc[0][i].x += m[i].x;
          acc[0][i].y += m[i].y;
        }
      }
    } else {
#pragma unroll 4
    for (int cp = 0; cp < CIN; ++cp) {
      float2 v[3], t[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) v[i] = __ldg(src + cp * 3 + i);
      if (d) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          t[i] = make_float2(0.f, 0.f);
#pragma unroll
          for (int j = 0; j < 3; ++j) cmac(t[i], w[3 * i + j], v[j]);
        }
      } else {
#pragma unroll
        for (int i = 0; i < 3; ++i) t[i] = v[i];
      }
      const float* wr = sw + (d * COUT) * CIN + cp;
#pragma unroll
      for (int c = 0; c < COUT; ++c) {
        const float k = wr[c * CIN];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          acc[c][i].x = fmaf(k, t[i].x, acc[c][i].x);
          acc[c][i].y = fmaf(k, t[i].y, acc[c][i].y);
        }
      }
    }
    }
  }
  if constexpr (COUT == 16) {
    // staged epilogue: the block's 128 sites x 16 channels go through shared
    // memory so that consecutive threads store consecutive 24-byte channel
    // vectors (a site's record is 384 bytes; per-site stores would be strided)
    extern __shared__ float net_epi[];  // [blockDim][97]
    float* e = net_epi + threadIdx.x * 97;
#pragma unroll
    for (int c = 0; c < 16; ++c)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        e[c * 6 + 2 * i] = acc[c][i].x;
        e[c * 6 + 2 * i + 1] = acc[c][i].y;
      }
    __syncthreads();
    const int base = blockIdx.x * blockDim.x;
    for (int q = threadIdx.x; q < (int)blockDim.x * 16; q += blockDim.x) {
      const int sl = q >> 4, c = q & 15, site = base + sl;
      if (site >= 2 * Vh) continue;
      const float* ev = net_epi + sl * 97 + c * 6;
      float2 v[3] = {make_float2(ev[0], ev[1]), make_float2(ev[2], ev[3]), make_float2(ev[4], ev[5])};
      float2* ho = hout + ((size_t)site * 16 + c) * 3;
      if (GATE) {
        const float n2 = v[0].x * v[0].x + v[0].y * v[0].y + v[1].x * v[1].x + v[1].y * v[1].y + v[2].x * v[2].x +
                         v[2].y * v[2].y;
        const float sg = 1.f / (1.f + __expf(-(n2 - bias[c])));
        float2* po = pre + ((size_t)site * 16 + c) * 3;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          po[i] = v[i];
          ho[i] = make_float2(v[i].x * sg, v[i].y * sg);
        }
      } else {
#pragma unroll
        for (int i = 0; i < 3; ++i) ho[i] = v[i];
      }
    }
    return;
  }
  if (!valid) return;
  float2* po = act_ptr(pre, COUT, Vh, p, s);
  float2* ho = act_ptr(hout, COUT, Vh, p, s);
#pragma unroll
  for (int c = 0; c < COUT; ++c) {
    if (GATE) {
      float n2 = 0.f;
#pragma unroll
      for (int i = 0; i < 3; ++i) n2 += acc[c][i].x * acc[c][i].x + acc[c][i].y * acc[c][i].y;
      const float sg = 1.f / (1.f + __expf(-(n2 - bias[c])));
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        po[c * 3 + i] = acc[c][i];
        ho[c * 3 + i] = make_float2(acc[c][i].x * sg, acc[c][i].y * sg);
      }
    } else {
#pragma unroll
      for (int i = 0; i < 3; ++i) ho[c * 3 + i] = acc[c][i];
    }
  }
}

// Gate backward: G_pre = s G_out + 2 s(1-s) Re<G_out, pre> pre  (in place on g)
// and per-block partial sums of db_c = -sum s(1-s) Re<G_out, pre>.  One
// thread per (site, channel): consecutive threads read and write consecutive
// 24-byte channel vectors; a thread's channel stays fixed over the
// grid-stride loop (the stride is a multiple of C).
template <int C>
__global__ void __launch_bounds__(256) k_net_gate_bwd(int n2vh, const float2* __restrict__ pre, float2* g,
                                                     const float* __restrict__ bias, float* __restrict__ db_part) {
  static_assert(C == 16, "one warp covers two sites of 16 channels");
  __shared__ float sdb[8][C];
  const int stride = gridDim.x * blockDim.x;
  const int q0 = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = q0 & (C - 1);
  const float bc = bias[c];
  float db = 0.f;
  for (int q = q0; q < n2vh * C; q += stride) {
    const float2* pv = pre + (size_t)q * 3;
    float2* gv = g + (size_t)q * 3;
    float2 v[3], o[3];
    float n2 = 0.f, pr = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      v[i] = pv[i];
      o[i] = gv[i];
      n2 += v[i].x * v[i].x + v[i].y * v[i].y;
      pr += o[i].x * v[i].x + o[i].y * v[i].y;
    }
    const float sg = 1.f / (1.f + __expf(-(n2 - bc)));
    const float sp = sg * (1.f - sg);
    db -= sp * pr;
#pragma unroll
    for (int i = 0; i < 3; ++i)
      gv[i] = make_float2(sg * o[i].x + 2.f * sp * pr * v[i].x, sg * o[i].y + 2.f * sp * pr * v[i].y);
  }
  // lanes l and l + 16 hold the same channel; then warps in order
  db += __shfl_xor_sync(0xffffffffu, db, 16);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane < C) sdb[warp][lane] = db;
  __syncthreads();
  if (threadIdx.x < C) {
    float v = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sdb[w][threadIdx.x];
    db_part[(size_t)blockIdx.x * C + threadIdx.x] = v;
  }
}

// Output layer with one channel, mix first: u_d(y) = sum_c' W[d][0][c'] h_c'(y)
// for the nine directions at every site (site-local, read once), then
// (see k_net_transport_sum) out(x) = sum_d (T_d u_d)(x).  U: [9][2 Vh][3].
template <int CIN>
__global__ void __launch_bounds__(256) k_net_mix_local(int n2vh, const float2* __restrict__ hin,
                                                      const __nv_bfloat16* __restrict__ W, float2* __restrict__ U) {
  __shared__ float sw[NET_NDIR * CIN];
  for (int i = threadIdx.x; i < NET_NDIR * CIN; i += blockDim.x) sw[i] = __bfloat162float(W[i]);
  __syncthreads();
  for (int site = blockIdx.x * blockDim.x + threadIdx.x; site < n2vh; site += gridDim.x * blockDim.x) {
    float2 u[NET_NDIR][3];
#pragma unroll
    for (int d = 0; d < NET_NDIR; ++d)
#pragma unroll
      for (int i = 0; i < 3; ++i) u[d][i] = make_float2(0.f, 0.f);
    const float4* src = (const float4*)(hin + (size_t)site * CIN * 3);
#pragma unroll
    for (int k = 0; k < CIN * 3 / 2; ++k) {  // float4 k holds entries 2k, 2k + 1 (channel e / 3, colour e % 3)
      const float4 f = __ldg(src + k);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int e = 2 * k + h, cp = e / 3, i = e - 3 * cp;
        const float vx = h ? f.z : f.x, vy = h ? f.w : f.y;
#pragma unroll
        for (int d = 0; d < NET_NDIR; ++d) {
          const float w = sw[d * CIN + cp];
          u[d][i].x = fmaf(w, vx, u[d][i].x);
          u[d][i].y = fmaf(w, vy, u[d][i].y);
        }
      }
    }
#pragma unroll
    for (int d = 0; d < NET_NDIR; ++d)
#pragma unroll
      for (int i = 0; i < 3; ++i) U[((size_t)d * n2vh + site) * 3 + i] = u[d][i];
  }
}

// out(x) = u_0(x) + sum_{d >= 1} hop_d(x) u_d(neighbour_d(x)).
__global__ void __launch_bounds__(256) k_net_transport_sum(NetGeom ng, const float2* __restrict__ U,
                                                          float2* __restrict__ hout) {
  const int Vh = ng.g.Vh, n2 = 2 * Vh;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n2; idx += gridDim.x * blockDim.x) {
    const int p = idx / Vh, s = idx - p * Vh;
    float2 acc[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) acc[i] = __ldg(U + (size_t)idx * 3 + i);
#pragma unroll 1
    for (int d = 1; d < NET_NDIR; ++d) {
      int np, ns;
      net_neighbour(ng, p, s, d, np, ns);
      float2 w[9], v[3];
      load_hop_matrix(ng, p, s, d, w);
      const float2* src = U + ((size_t)d * n2 + (size_t)np * Vh + ns) * 3;
#pragma unroll
      for (int j = 0; j < 3; ++j) v[j] = __ldg(src + j);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) cmac(acc[i], w[3 * i + j], v[j]);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) hout[(size_t)idx * 3 + i] = acc[i];
  }
}

// Weight gradient: dW[d][c][c'] = sum_x Re<G_pre_c(x), (T_d h_c')(x)>.
// A block stages a tile of TS sites: the 9 transports of every input channel
// and the output gradients, in shared memory; then thread (d, tile of 4x4
// (c, c') pairs) accumulates over the tile's sites.  Per-block sums go to
// part[block][9*COUT*CIN] (a fixed-order final sum follows).
template <int CIN, int COUT, int TS>
__global__ void __launch_bounds__(256) k_net_dw(NetGeom ng, const float2* __restrict__ hin,
                                               const float2* __restrict__ g, float* __restrict__ part) {
  constexpr int TC = (COUT + 3) / 4, TP = (CIN + 3) / 4;  // 4x4 tiles
  constexpr int NT = NET_NDIR * TC * TP;                  // accumulating threads
  extern __shared__ float smem[];
  float* st = smem;                                  // [TS][9][CIN][6]
  float* sg = smem + TS * NET_NDIR * CIN * 6;        // [TS][COUT][6]
  const int Vh = ng.g.Vh;
  const int n2 = 2 * Vh;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  const int tid = threadIdx.x;
  const int td = tid / (TC * TP), tr = tid % (TC * TP), tc = tr / TP, tp = tr % TP;
  for (int base = blockIdx.x * TS; base < n2; base += gridDim.x * TS) {
    __syncthreads();
    // stage transports: item = (site in tile, d, channel)
    for (int it = tid; it < TS * NET_NDIR * CIN; it += blockDim.x) {
      const int ls = it / (NET_NDIR * CIN), rem = it % (NET_NDIR * CIN), d = rem / CIN, cp = rem % CIN;
      const int site = base + ls;
      float2 t[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      if (site < n2) {
        const int p = site / Vh, s = site - p * Vh;
        int np, ns;
        net_neighbour(ng, p, s, d, np, ns);
        const float2* src = act_ptr(hin, CIN, Vh, np, ns) + cp * 3;
        float2 v[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) v[i] = __ldg(src + i);
        if (d) {
          float2 w[9];
          load_hop_matrix(ng, p, s, d, w);
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) cmac(t[i], w[3 * i + j], v[j]);
        } else {
#pragma unroll
          for (int i = 0; i < 3; ++i) t[i] = v[i];
        }
      }
      float* dst = st + ((ls * NET_NDIR + d) * CIN + cp) * 6;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        dst[2 * i] = t[i].x;
        dst[2 * i + 1] = t[i].y;
      }
    }
    for (int it = tid; it < TS * COUT * 6; it += blockDim.x) {
      const int ls = it / (COUT * 6), rem = it % (COUT * 6);
      const int site = base + ls;
      sg[it] = site < n2 ? ((const float*)(g + (size_t)site * COUT * 3))[rem] : 0.f;
    }
    __syncthreads();
    if (tid < NT) {
      for (int ls = 0; ls < TS; ++ls) {
        const float* tv = st + (ls * NET_NDIR + td) * CIN * 6;
        const float* gv = sg + ls * COUT * 6;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          float ga[4], tb[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) ga[a] = (tc * 4 + a < COUT) ? gv[(tc * 4 + a) * 6 + i] : 0.f;
#pragma unroll
          for (int b = 0; b < 4; ++b) tb[b] = (tp * 4 + b < CIN) ? tv[(tp * 4 + b) * 6 + i] : 0.f;
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(ga[a], tb[b], acc[a][b]);
        }
      }
    }
  }
  if (tid < NT) {
    float* out = part + (size_t)blockIdx.x * NET_NDIR * COUT * CIN;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int c = tc * 4 + a, cp = tp * 4 + b;
        if (c < COUT && cp < CIN) out[(td * COUT + c) * CIN + cp] = acc[a][b];
      }
  }
}

// grad[i] += sum over blocks of part[block][i] (fixed block order)
__global__ void k_net_sum_parts(const float* __restrict__ part, int nblocks, int n, float* grad) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * n + i];
    grad[i] += s;
  }
}

}  // namespace stag
