// a4 distributed over a thread-block cluster: Algorithm 4 for one OCP whose workspace does not
// fit in one CTA's shared memory (12-state rigid body, T up to a few hundred).  CTA 0 of the
// cluster (the leader) runs every other stage of the SQP iteration and the backward pass from the
// OCP's global-memory workspace, as the single-team kernel does.  At each PCG solve it hands the
// solve to all CTAs of the cluster: CTA r copies the knots [r KC, (r+1) KC) of the S and Phi^-1
// blocks, the factors A_t, B_t and the FP64 vectors into its own shared memory, and the PCG then
// runs with every block resident on chip:
//   - knot k's row of S p (and of Phi^-1 r) needs p_{k-1} and the product with block k+1; a CTA
//     keeps the first block of the next CTA as a halo copy, and the owner of a boundary knot
//     pushes the vector values its neighbours need into their shared memory (DSMEM stores)
//     before the next all-reduce, so no extra synchronisation is needed for the halos;
//   - each of the two dot products of an iteration is an all-reduce: warp shuffles, one partial
//     per warp, then every CTA stores its partial into a slot of every other CTA and arrives on
//     that CTA's mbarrier; every CTA sums the slots in rank order, so all CTAs hold bitwise the
//     same totals and take the same decisions;
//   - reliable updates evaluate the FP64 true residual gamma - H G^-1 H^T lambda from the
//     factors (hp_apply's two passes, distributed the same way) and the stagnation test hands
//     the solve back to the leader, which finishes it with the double-float rescue from global
//     memory, exactly as the single-team kernel does.
// Every wait on another CTA is an mbarrier wait with a time limit; when one runs out the CTA
// stops waiting from then on, and the OCP is flagged (ST_SYNC_TIMEOUT).
#pragma once
#include "cluster.cuh"

namespace dmpc {

constexpr int kClMaxCtas = 8;     // CTAs per cluster (the portable cluster size)
constexpr int kClThreads = 256;   // threads per CTA (the leader's team)
constexpr int kClRows = 2;        // rows of a knot's block row per thread
constexpr int kClNV = 2;          // widest all-reduce
constexpr unsigned long long kClWaitNs = 4000000000ull;  // time limit of one wait (4 s)
constexpr int ST_SYNC_TIMEOUT = 256;

#ifdef DMPC_CLUSTER_PCG
constexpr bool kClusterPcg = true;
#else
constexpr bool kClusterPcg = false;
#endif

enum ClCommand : int { CL_PCG = 1, CL_EXIT = 2 };

// Shared-memory layout of one CTA of the cluster (float offsets unless noted).  KC = knot
// capacity per CTA.  Blocks are knot-minor over KB = KC + 1 slots (slot KC + ... : the next
// CTA's first knot); vectors over KV = KC + 2 slots: slot 0 = the previous CTA's last knot,
// slots 1..nk = own knots, slot nk + 1 = the next CTA's first knot.
struct ClLayout {
  int KC, KB, KV;
  int D, O, Pd, Po, A, Bm;   // float blocks
  int Pv, R, Y, Z, DL;       // float vectors
  int rh, yh, zh, ph;        // halo staging, [side][NX]: side 0 = previous CTA, 1 = next CTA
  int misc;                  // copy of the OCP's scalars (weights, reciprocals)
  int wpart, slots;          // all-reduce scratch: 2 x warps x kClNV, 2 x kClMaxCtas x kClNV
  int job;                   // command words written by the leader
  int bars;                  // mbarriers (8 bytes each): all-reduce 0, 1, command
  int dbase;                 // float offset of the double region
  int LP, G, WX, WU;         // double vectors (offsets in doubles from dbase)
  int total;
};

__host__ __device__ inline ClLayout cl_layout(int nx, int nu, int kc) {
  ClLayout S;
  S.KC = kc;
  S.KB = kc + 1;
  S.KV = kc + 2;
  int f = 0;
  const int b = nx * nx * S.KB;
  S.D = f; f += b;
  S.O = f; f += b;
  S.Pd = f; f += b;
  S.Po = f; f += b;
  S.A = f; f += b;
  S.Bm = f; f += nx * nu * S.KB;
  const int v = nx * S.KV;
  S.Pv = f; f += v;
  S.R = f; f += v;
  S.Y = f; f += v;
  S.Z = f; f += v;
  S.DL = f; f += v;
  S.rh = f; f += 2 * nx;
  S.yh = f; f += 2 * nx;
  S.zh = f; f += 2 * nx;
  S.ph = f; f += 2 * nx;
  f = (f + 3) & ~3;
  S.misc = f; f += kMisc;
  S.wpart = f; f += 2 * (kClThreads / 32) * kClNV;
  S.slots = f; f += 2 * kClMaxCtas * kClNV;
  S.job = f; f += 8;
  f = (f + 3) & ~3;
  S.bars = f; f += 8;
  S.dbase = f;
  int d = 0;
  S.LP = d; d += nx * S.KV;
  S.G = d; d += nx * S.KV;
  S.WX = d; d += nx * S.KV;
  S.WU = d; d += nu * S.KV;
  f += 2 * d;
  S.total = (f + 3) & ~3;
  return S;
}

// Largest knot count per CTA: one thread per (knot, group of kClRows rows).
__host__ __device__ constexpr int cl_max_kc(int nx) { return kClThreads / (nx / kClRows); }

// Per-thread state of the distributed PCG in one CTA.
template <class M>
struct ClRun {
  static constexpr int NX = M::NX, NU = M::NU, RG = NX / kClRows;
  float* sm;
  double* dm;
  ClLayout S;
  uint32_t rank, ncta;
  int tid;
  int phase;        // all-reduce phase counter
  uint32_t cmd_par; // parity of the next command phase (followers)
  bool broken;      // a wait ran out: no more waiting in this CTA
  // current OCP
  int K, T, KC, k0, nk, kl, r0;
  bool act, has_prev, has_next;

  __device__ __forceinline__ float* F(int off) const { return sm + off; }
  __device__ __forceinline__ double* Dd(int off) const { return dm + off; }
  __device__ __forceinline__ uint32_t bar(int i) const { return cl::saddr(sm + S.bars) + 8u * (uint32_t)i; }
  __device__ __forceinline__ double qinv(int k, int i) const {
    return reinterpret_cast<const double*>(sm + S.misc + MS_DINV)[(k < T ? 0 : 24) + i];
  }
  __device__ __forceinline__ double rinv(int i) const {
    return reinterpret_cast<const double*>(sm + S.misc + MS_DINV)[16 + i];
  }
  // shared::cluster address of element `off` (floats) of CTA `r`'s shared memory
  __device__ __forceinline__ uint32_t remote(int off, uint32_t r) const { return cl::map(cl::saddr(sm + off), r); }
  __device__ __forceinline__ uint32_t remote_d(int doff, uint32_t r) const {
    return cl::map(cl::saddr(dm + doff), r);
  }

  __device__ void init(float* smem, int kc) {
    sm = smem;
    S = cl_layout(NX, NU, kc);
    dm = reinterpret_cast<double*>(smem + S.dbase);
    rank = cl::rank();
    ncta = cl::ncta();
    tid = threadIdx.x;
    phase = 0;
    cmd_par = 0;
    broken = false;
  }
  // knot partition of an OCP with K knots over the cluster's CTAs
  __device__ void bind(int K_, int T_) {
    K = K_;
    T = T_;
    KC = (K + (int)ncta - 1) / (int)ncta;
    k0 = (int)rank * KC;
    nk = K - k0;
    nk = nk < 0 ? 0 : (nk > KC ? KC : nk);
    act = nk > 0 && tid < RG * nk;
    kl = act ? tid % nk : 0;
    r0 = act ? (tid / nk) * kClRows : 0;
    has_prev = nk > 0 && k0 > 0;
    has_next = nk > 0 && k0 + nk < K;
  }
};

// Sum NV values over every thread of every CTA of the cluster; all threads of all CTAs receive
// bitwise the same totals.  Also a cluster-wide barrier: shared-memory and global writes made
// before it by any thread of the cluster are visible after it.
template <class M, int NV>
__device__ __forceinline__ void cl_sum(ClRun<M>& r, float (&v)[NV]) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] += __shfl_xor_sync(0xffffffffu, v[j], off);
  }
  const int b = r.phase & 1;
  const uint32_t par = (uint32_t)(r.phase >> 1) & 1u;
  float* wp = r.F(r.S.wpart) + b * (kClThreads / 32) * kClNV;
  float* sl = r.F(r.S.slots) + b * kClMaxCtas * kClNV;
  if ((r.tid & 31) == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) wp[(r.tid >> 5) * kClNV + j] = v[j];
  }
  __syncthreads();
  if (r.tid < (int)r.ncta && !r.broken) {
    float s[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) s[j] = 0.f;
    for (int q = 0; q < kClThreads / 32; ++q) {
#pragma unroll
      for (int j = 0; j < NV; ++j) s[j] += wp[q * kClNV + j];
    }
    const uint32_t dst = r.remote(r.S.slots + b * kClMaxCtas * kClNV + (int)r.rank * kClNV, (uint32_t)r.tid);
#pragma unroll
    for (int j = 0; j < NV; ++j) cl::st_f32(dst + 4u * (uint32_t)j, s[j]);
    cl::arrive_remote(cl::map(r.bar(b), (uint32_t)r.tid));
  }
  bool ok = r.broken ? false : cl::wait(r.bar(b), par, kClWaitNs);
  ok = __syncthreads_and(ok) != 0;
  if (!ok) r.broken = true;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    float t = 0.f;
    for (uint32_t q = 0; q < r.ncta; ++q) t += sl[q * kClNV + j];
    v[j] = t;
  }
  ++r.phase;
}

template <class M>
__device__ __forceinline__ void cl_barrier(ClRun<M>& r) {
  float d[1] = {0.f};
  cl_sum<M, 1>(r, d);
}

// Push this thread's rows of a boundary knot's values into the staging arrays of the
// neighbouring CTAs (side 1 of the previous CTA, side 0 of the next CTA).
template <class M>
__device__ __forceinline__ void cl_push_pair(ClRun<M>& r, int st_a, int st_b, const float* a, const float* b) {
  constexpr int NX = M::NX;
  if (!r.act) return;
  if (r.kl == 0 && r.has_prev) {
    const uint32_t da = r.remote(st_a + NX + r.r0, r.rank - 1), db = r.remote(st_b + NX + r.r0, r.rank - 1);
#pragma unroll
    for (int q = 0; q < kClRows; ++q) { cl::st_f32(da + 4u * q, a[q]); cl::st_f32(db + 4u * q, b[q]); }
  }
  if (r.kl == r.nk - 1 && r.has_next) {
    const uint32_t da = r.remote(st_a + r.r0, r.rank + 1), db = r.remote(st_b + r.r0, r.rank + 1);
#pragma unroll
    for (int q = 0; q < kClRows; ++q) { cl::st_f32(da + 4u * q, a[q]); cl::st_f32(db + 4u * q, b[q]); }
  }
}

// Rows [r0, r0 + kClRows) of the symmetric block-tridiagonal row of knot kl:
// out = Md_k v_k + Mo_k v_{k-1} + Mo_{k+1}^T v_{k+1} (block slots kl and kl + 1, vector slots
// kl, kl + 1, kl + 2; missing neighbours are zero blocks and zero halos).
template <class M, class V>
__device__ __forceinline__ void cl_btmv_rows(const ClRun<M>& r, int md, int mo, const V* v, float (&out)[kClRows]) {
  constexpr int NX = M::NX;
  const int KB = r.S.KB, KV = r.S.KV, kl = r.kl;
  const float* Md = r.F(md);
  const float* Mo = r.F(mo);
  float vm[NX], vc[NX], vp[NX];
#pragma unroll
  for (int j = 0; j < NX; ++j) {
    vm[j] = (float)v[j * KV + kl];
    vc[j] = (float)v[j * KV + kl + 1];
    vp[j] = (float)v[j * KV + kl + 2];
  }
#pragma unroll
  for (int q = 0; q < kClRows; ++q) {
    const int i = r.r0 + q;
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < NX; ++j) acc = fmaf(Md[(i * NX + j) * KB + kl], vc[j], acc);
#pragma unroll
    for (int j = 0; j < NX; ++j) acc = fmaf(Mo[(i * NX + j) * KB + kl], vm[j], acc);
#pragma unroll
    for (int j = 0; j < NX; ++j) acc = fmaf(Mo[(j * NX + i) * KB + kl + 1], vp[j], acc);
    out[q] = acc;
  }
}

// Z = Phi^-1 R on this thread's rows; returns its share of R^T Z and pushes the boundary knots'
// z and p to the neighbours (for their p halo after the next all-reduce).
template <class M>
__device__ __forceinline__ float cl_precond(ClRun<M>& r) {
  constexpr int NX = M::NX;
  if (!r.act) return 0.f;
  const int KV = r.S.KV, s = r.kl + 1;
  float z[kClRows], pv[kClRows];
  cl_btmv_rows<M, float>(r, r.S.Pd, r.S.Po, r.F(r.S.R), z);
  float e = 0.f;
#pragma unroll
  for (int q = 0; q < kClRows; ++q) {
    const int i = r.r0 + q;
    r.F(r.S.Z)[i * KV + s] = z[q];
    e = fmaf(r.F(r.S.R)[i * KV + s], z[q], e);
    pv[q] = r.F(r.S.Pv)[i * KV + s];
  }
  (void)NX;
  cl_push_pair<M>(r, r.S.zh, r.S.ph, z, pv);
  return e;
}

// FP64 true residual R = gamma - H G^-1 H^T LP on the own knots (hp_apply's two passes), leaving
// WX, WU = H^T LP; halos: the next CTA's first LP (pushed when push_lp, else already present),
// the previous CTA's last WX, WU and both neighbours' new R (pushed).
template <class M>
__device__ void cl_hp_residual(ClRun<M>& r, bool push_lp) {
  constexpr int NX = M::NX, NU = M::NU;
  const int KB = r.S.KB, KV = r.S.KV, kl = r.kl, s = kl + 1;
  const int k = r.k0 + kl;
  double* LP = r.Dd(r.S.LP);
  double* WX = r.Dd(r.S.WX);
  double* WU = r.Dd(r.S.WU);
  const double* G = r.Dd(r.S.G);
  const float* A = r.F(r.S.A);
  const float* Bm = r.F(r.S.Bm);
  if (push_lp) {
    if (r.act && kl == 0 && r.has_prev) {
#pragma unroll
      for (int q = 0; q < kClRows; ++q) {
        const int i = r.r0 + q;
        cl::st_f64(r.remote_d(r.S.LP + i * KV + r.KC + 1, r.rank - 1), LP[i * KV + s]);
      }
    }
    cl_barrier<M>(r);
  }
  // pass 1: w = H^T LP at knot k (A_k, B_k at block slot kl + 1, stored as A_k + I)
  if (r.act) {
    double ln[NX];
#pragma unroll
    for (int j = 0; j < NX; ++j) ln[j] = (k < r.T) ? LP[j * KV + s + 1] : 0.0;
    double wx[kClRows];
#pragma unroll
    for (int q = 0; q < kClRows; ++q) {
      const int i = r.r0 + q;
      double acc = LP[i * KV + s];
      if (k < r.T) {
        acc -= ln[i];
#pragma unroll
        for (int j = 0; j < NX; ++j) acc += (double)A[(j * NX + i) * KB + kl + 1] * ln[j];
      }
      wx[q] = acc;
      WX[i * KV + s] = acc;
    }
    for (int u = r.r0 / kClRows; u < NU; u += r.RG) {
      double acc = 0.0;
      if (k < r.T) {
#pragma unroll
        for (int j = 0; j < NX; ++j) acc += (double)Bm[(j * NU + u) * KB + kl + 1] * ln[j];
      }
      WU[u * KV + s] = acc;
      if (kl == r.nk - 1 && r.has_next) cl::st_f64(r.remote_d(r.S.WU + u * KV + 0, r.rank + 1), acc);
    }
    if (kl == r.nk - 1 && r.has_next) {
#pragma unroll
      for (int q = 0; q < kClRows; ++q)
        cl::st_f64(r.remote_d(r.S.WX + (r.r0 + q) * KV + 0, r.rank + 1), wx[q]);
    }
  }
  cl_barrier<M>(r);
  // pass 2: (H G^-1 w)_k on this thread's rows, then R = gamma - that
  if (r.act) {
    float rv[kClRows], zero[kClRows];
    double vx[NX], vu[NU];
    if (k > 0) {
#pragma unroll
      for (int j = 0; j < NX; ++j) vx[j] = WX[j * KV + s - 1] * r.qinv(k - 1, j);
#pragma unroll
      for (int j = 0; j < NU; ++j) vu[j] = WU[j * KV + s - 1] * r.rinv(j);
    }
#pragma unroll
    for (int q = 0; q < kClRows; ++q) {
      const int i = r.r0 + q;
      double acc = WX[i * KV + s] * r.qinv(k, i);
      if (k > 0) {
        acc -= vx[i];
#pragma unroll
        for (int j = 0; j < NX; ++j) acc += (double)A[(i * NX + j) * KB + kl] * vx[j];
#pragma unroll
        for (int j = 0; j < NU; ++j) acc += (double)Bm[(i * NU + j) * KB + kl] * vu[j];
      }
      rv[q] = (float)(G[i * KV + s] - acc);
      r.F(r.S.R)[i * KV + s] = rv[q];
      zero[q] = 0.f;
    }
    cl_push_pair<M>(r, r.S.rh, r.S.yh, rv, zero);
  }
  cl_barrier<M>(r);
  // R halos from the pushed values
  if (r.tid < 2 * NX) {
    const int side = r.tid / NX, i = r.tid % NX;
    if (side == 0 ? r.has_prev : r.has_next)
      r.F(r.S.R)[i * KV + (side == 0 ? 0 : r.nk + 1)] = r.F(r.S.rh)[side * NX + i];
  }
  __syncthreads();
}

struct ClResult {
  int it;
  bool converged;
  float eta0;
};

// The distributed PCG of one OCP, run by every CTA of the cluster.  ws: the OCP's global
// workspace (leader's layout L).  On return LP (the solution) and WX, WU (= H^T LP) are back in
// the global workspace.
template <class M>
__device__ ClResult cl_pcg(ClRun<M>& r, const KParams& P, int K, int T, float* ws) {
  constexpr int NX = M::NX, NU = M::NU;
  ClResult res{0, false, 0.f};
  r.bind(K, T);
  const Layout L = make_layout(NX, NU, K, kClThreads, P.opt.exact_hessian, 0);
  const int KP = L.KP, KB = r.S.KB, KV = r.S.KV, nk = r.nk, k0 = r.k0;
  const double* wd = reinterpret_cast<const double*>(ws);
  // stage the blocks (own knots and the next CTA's first knot) and vectors from global memory;
  // missing neighbours and the unused slot-0 blocks (O_0, Phi^-1 off-diagonal, A, B at k = 0)
  // are zero
  {
    const int nb = nk + 1;
    const int offs[5] = {L.D, L.O, L.Pd, L.Po, L.A};
    const int so[5] = {r.S.D, r.S.O, r.S.Pd, r.S.Po, r.S.A};
    for (int a = 0; a < 5; ++a) {
      for (int idx = r.tid; idx < NX * NX * nb; idx += kClThreads) {
        const int e = idx / nb, j = idx % nb, k = k0 + j;
        const bool zero_at0 = (a == 1 || a == 3 || a == 4) && k == 0;
        r.sm[so[a] + e * KB + j] = (nk > 0 && k < K && !zero_at0) ? __ldcg(ws + offs[a] + e * KP + k) : 0.f;
      }
    }
    for (int idx = r.tid; idx < NX * NU * nb; idx += kClThreads) {
      const int e = idx / nb, j = idx % nb, k = k0 + j;
      r.sm[r.S.Bm + e * KB + j] = (nk > 0 && k < K && k > 0) ? __ldcg(ws + L.Bm + e * KP + k) : 0.f;
    }
    for (int idx = r.tid; idx < NX * KV; idx += kClThreads) {
      const int i = idx / KV, sl = idx % KV, k = k0 + sl - 1;
      const bool in = nk > 0 && sl <= nk + 1 && k >= 0 && k < K;
      r.Dd(r.S.LP)[idx] = in ? __ldcg(wd + L.d_lamp + i * KP + k) : 0.0;
      r.Dd(r.S.G)[idx] = in ? __ldcg(wd + L.d_gam + i * KP + k) : 0.0;
      r.Dd(r.S.WX)[idx] = 0.0;
      r.F(r.S.Pv)[idx] = 0.f;
      r.F(r.S.R)[idx] = 0.f;
      r.F(r.S.Y)[idx] = 0.f;
      r.F(r.S.Z)[idx] = 0.f;
      r.F(r.S.DL)[idx] = 0.f;
    }
    for (int idx = r.tid; idx < NU * KV; idx += kClThreads) r.Dd(r.S.WU)[idx] = 0.0;
    for (int idx = r.tid; idx < kMisc; idx += kClThreads) r.sm[r.S.misc + idx] = __ldcg(ws + L.misc + idx);
    for (int idx = r.tid; idx < 8 * NX; idx += kClThreads) r.sm[r.S.rh + idx] = 0.f;  // rh, yh, zh, ph
  }
  __syncthreads();
  const float tol2 = P.opt.pcg_tol * P.opt.pcg_tol;
  const float dl2 = P.opt.ru_delta * P.opt.ru_delta;
  const int maxit = P.opt.pcg_max_iters;
  float* Pv = r.F(r.S.Pv);
  float* R = r.F(r.S.R);
  float* Y = r.F(r.S.Y);
  float* Z = r.F(r.S.Z);
  float* DL = r.F(r.S.DL);
  double* LP = r.Dd(r.S.LP);
  const int s = r.kl + 1;

  // true residual of the initial guess (its next-CTA LP halo came from global memory)
  cl_hp_residual<M>(r, false);
  float e0[2] = {0.f, 0.f};
  if (r.act) {
    e0[0] = cl_precond<M>(r);
    float gt[kClRows];
    cl_btmv_rows<M, double>(r, r.S.Pd, r.S.Po, r.Dd(r.S.G), gt);
#pragma unroll
    for (int q = 0; q < kClRows; ++q) e0[1] = fmaf((float)r.Dd(r.S.G)[(r.r0 + q) * KV + s], gt[q], e0[1]);
  }
  cl_sum<M, 2>(r, e0);
  float eta = e0[0];
  const float eta0 = e0[1];
  res.eta0 = eta0;
  // p = z (beta = 0): own rows and halos
  auto update_p = [&](float beta) {
    if (r.tid < 2 * NX) {
      const int side = r.tid / NX, i = r.tid % NX;
      if (side == 0 ? r.has_prev : r.has_next)
        Pv[i * KV + (side == 0 ? 0 : nk + 1)] = fmaf(beta, r.F(r.S.ph)[side * NX + i], r.F(r.S.zh)[side * NX + i]);
    }
    if (r.act) {
#pragma unroll
      for (int q = 0; q < kClRows; ++q) {
        const int i = r.r0 + q;
        Pv[i * KV + s] = fmaf(beta, Pv[i * KV + s], Z[i * KV + s]);
      }
    }
    __syncthreads();
  };
  update_p(0.f);
  float eta_ref = eta, eta_true = eta;
  int it = 0, stall = 0;
  bool converged = !(eta > tol2 * eta0);
  bool folded = true;
  while (!converged && it < maxit && !r.broken) {
    // y = S p, v = p^T y; boundary knots push their r and y for the neighbours' r halo
    float v[1] = {0.f};
    if (r.act) {
      float y[kClRows], rv[kClRows];
      cl_btmv_rows<M, float>(r, r.S.D, r.S.O, Pv, y);
#pragma unroll
      for (int q = 0; q < kClRows; ++q) {
        const int i = r.r0 + q;
        Y[i * KV + s] = y[q];
        v[0] = fmaf(Pv[i * KV + s], y[q], v[0]);
        rv[q] = R[i * KV + s];
      }
      cl_push_pair<M>(r, r.S.rh, r.S.yh, rv, y);
    }
    cl_sum<M, 1>(r, v);
    if (!(v[0] > 0.f) || !isfinite(v[0])) break;
    const float alpha = eta / v[0];
    if (r.act) {
#pragma unroll
      for (int q = 0; q < kClRows; ++q) {
        const int i = r.r0 + q;
        DL[i * KV + s] = fmaf(alpha, Pv[i * KV + s], DL[i * KV + s]);
        R[i * KV + s] = fmaf(-alpha, Y[i * KV + s], R[i * KV + s]);
      }
    }
    if (r.tid < 2 * NX) {
      const int side = r.tid / NX, i = r.tid % NX;
      if (side == 0 ? r.has_prev : r.has_next)
        R[i * KV + (side == 0 ? 0 : nk + 1)] = fmaf(-alpha, r.F(r.S.yh)[side * NX + i], r.F(r.S.rh)[side * NX + i]);
    }
    folded = false;
    __syncthreads();
    float e1[1] = {cl_precond<M>(r)};
    cl_sum<M, 1>(r, e1);
    float eta_new = e1[0];
    ++it;
    if (eta_new < dl2 * eta_ref || !(eta_new > tol2 * eta0) || it >= maxit || !isfinite(eta_new)) {
      // reliable update: fold the FP32 correction into the FP64 solution, true residual
      if (r.act) {
#pragma unroll
        for (int q = 0; q < kClRows; ++q) {
          const int i = r.r0 + q;
          LP[i * KV + s] += (double)DL[i * KV + s];
          DL[i * KV + s] = 0.f;
        }
      }
      folded = true;
      cl_hp_residual<M>(r, true);
      float e2[1] = {cl_precond<M>(r)};
      cl_sum<M, 1>(r, e2);
      eta_new = e2[0];
      eta_ref = eta_new;
      if (!(eta_new > tol2 * eta0)) { converged = true; break; }
      if (!isfinite(eta_new)) break;
      if (eta_new > 0.25f * eta_true) {
        if (++stall >= 2) break;
      } else {
        stall = 0;
      }
      eta_true = eta_new;
      if (it >= maxit) break;
    }
    const float beta = eta_new / eta;
    eta = eta_new;
    update_p(beta);
  }
  if (!folded && !r.broken) {
    if (r.act) {
#pragma unroll
      for (int q = 0; q < kClRows; ++q) {
        const int i = r.r0 + q;
        LP[i * KV + s] += (double)DL[i * KV + s];
      }
    }
    cl_hp_residual<M>(r, true);
  }
  // own knots of LP, WX, WU back to the global workspace
  if (!r.broken) {
    double* gd = reinterpret_cast<double*>(ws);
    for (int idx = r.tid; idx < NX * nk; idx += kClThreads) {
      const int i = idx / nk, j = idx % nk;
      gd[L.d_lamp + i * KP + k0 + j] = LP[i * KV + j + 1];
      gd[L.d_wx + i * KP + k0 + j] = r.Dd(r.S.WX)[i * KV + j + 1];
    }
    for (int idx = r.tid; idx < NU * nk; idx += kClThreads) {
      const int i = idx / nk, j = idx % nk;
      gd[L.d_wu + i * KP + k0 + j] = r.Dd(r.S.WU)[i * KV + j + 1];
    }
  }
  cl_barrier<M>(r);
  res.it = it;
  res.converged = converged && !r.broken;
  return res;
}

// Leader: send a command to the other CTAs of the cluster.  The team's earlier global-memory
// writes are released with it.
template <class M>
__device__ void cl_command(ClRun<M>& r, int cmd, int ocp, int K, int T) {
  __syncthreads();
  if (r.tid == 0) {
    int* job = reinterpret_cast<int*>(r.sm + r.S.job);
    job[0] = cmd; job[1] = ocp; job[2] = K; job[3] = T;
  }
  __syncthreads();
  if (r.tid >= 1 && r.tid < (int)r.ncta && !r.broken) cl::arrive_remote(cl::map(r.bar(2), (uint32_t)r.tid));
}

// Other CTAs: run the leader's PCG commands until it sends CL_EXIT (or a wait runs out).
template <class M>
__device__ void cl_follower(ClRun<M>& r, const KParams& P, float* ws) {
  while (!r.broken) {
    bool ok = cl::wait(r.bar(2), r.cmd_par, kClWaitNs);
    ok = __syncthreads_and(ok) != 0;
    if (!ok) { r.broken = true; break; }
    r.cmd_par ^= 1u;
    const uint32_t jb = r.remote(r.S.job, 0);
    const int cmd = cl::ld_s32(jb), K = cl::ld_s32(jb + 8), T = cl::ld_s32(jb + 12);
    if (cmd != CL_PCG) break;
    cl_pcg<M>(r, P, K, T, ws);
  }
}

}  // namespace dmpc
