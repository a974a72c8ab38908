// One timestep of Eq. general_ST_decomposition (Sec. 3, arXiv 1801.10233):
//   half-kick, spin half-op, drift (+ rebuild check, exchange table),
//   spin half-op, forces + half-kick.
// The spin half-op e^{Ls dt/2} is 8 colour passes forward then 8 backward
// (Eq. spin_ST_sectoring, Sec. 5.1); each pass updates every sector of one
// colour concurrently, the spins inside a sector one after another.
#include "sl_internal.cuh"

namespace {

inline int grid_for(int n) { return (n + SL_BLOCK - 1) / SL_BLOCK; }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11) and Box-Muller normals for the spin bath.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
    unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__device__ __forceinline__ double3 gauss3(uint64_t seed, int replica, long long step, int subpass, int atom) {
  uint4 x = philox4x32_10(make_uint4((unsigned)atom, (unsigned)step, (unsigned)subpass, (unsigned)replica),
                          make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
  const double inv32 = 2.3283064365386962890625e-10;  // 2^-32
  const double twopi = 6.283185307179586476925286766559;
  double u0 = ((double)x.x + 0.5) * inv32, u1 = ((double)x.y + 0.5) * inv32;
  double u2 = ((double)x.z + 0.5) * inv32, u3 = ((double)x.w + 0.5) * inv32;
  double ra = sqrt(-2.0 * log(u0)), rb = sqrt(-2.0 * log(u2));
  double s1, c1, s3, c3;
  sincos(twopi * u1, &s1, &c1);
  sincos(twopi * u3, &s3, &c3);
  return make_double3(ra * c1, ra * s1, rb * c3);
}

// ---------------------------------------------------------------------------
// Single-spin propagator e^{L_si tau}.
//
// Exact rotation of s about w by theta = |w| tau, written without |w| and as
// an increment of s so that each component is rounded once:
//   s' = s + [ -u B s + tau A (w x s) + tau^2 B (w.s) w ]
// with u = theta^2, A = sin(theta)/theta and B = (1 - cos(theta))/theta^2
// (so 1 - cos(theta) = u B).  A and B are even power series in theta; for
// theta <= 0.25 the Taylor series truncated after the u^6 term are exact to
// below 1e-17 relative.  Larger angles use sqrt and sincos.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void rotate_exact(double3 w, double tau, double4_32a& s) {
  double u = tau * tau * (w.x * w.x + w.y * w.y + w.z * w.z);
  double A, B, uB;
  if (u <= 0.0625) {
    // 1/(2k+1)! and 1/(2k+2)! for k = 0..6
    A = 1.0 / 6227020800.0;                 // 1/13!
    A = fma(A, -u, 1.0 / 39916800.0);       // 1/11!
    A = fma(A, -u, 1.0 / 362880.0);         // 1/9!
    A = fma(A, -u, 1.0 / 5040.0);           // 1/7!
    A = fma(A, -u, 1.0 / 120.0);            // 1/5!
    A = fma(A, -u, 1.0 / 6.0);              // 1/3!
    A = fma(A, -u, 1.0);
    B = 1.0 / 87178291200.0;                // 1/14!
    B = fma(B, -u, 1.0 / 479001600.0);      // 1/12!
    B = fma(B, -u, 1.0 / 3628800.0);        // 1/10!
    B = fma(B, -u, 1.0 / 40320.0);          // 1/8!
    B = fma(B, -u, 1.0 / 720.0);            // 1/6!
    B = fma(B, -u, 1.0 / 24.0);             // 1/4!
    B = fma(B, -u, 0.5);                    // 1/2!
    uB = u * B;
  } else {
    double th = sqrt(u);
    double h = sin(0.5 * th);
    A = sin(th) / th;
    uB = 2.0 * h * h;
    B = uB / u;
  }
  double tA = tau * A, tB = tau * tau * B * (w.x * s.x + w.y * s.y + w.z * s.z);
  double cx = w.y * s.z - w.z * s.y;
  double cy = w.z * s.x - w.x * s.z;
  double cz = w.x * s.y - w.y * s.x;
  double ix = fma(-uB, s.x, fma(tA, cx, tB * w.x));
  double iy = fma(-uB, s.y, fma(tA, cy, tB * w.y));
  double iz = fma(-uB, s.z, fma(tA, cz, tB * w.z));
  s.x += ix; s.y += iy; s.z += iz;
}

// Cayley-type propagator printed in Sec. 3 (rotation by 2 atan(|w| tau/2)).
__device__ __forceinline__ void rotate_cayley(double3 w, double tau, double4_32a& s) {
  double w2 = w.x * w.x + w.y * w.y + w.z * w.z;
  double ws = w.x * s.x + w.y * s.y + w.z * s.z;
  double q = 0.25 * tau * tau;
  double inv = 1.0 / (1.0 + q * w2);
  double cx = w.y * s.z - w.z * s.y;
  double cy = w.z * s.x - w.x * s.z;
  double cz = w.x * s.y - w.y * s.x;
  double x = s.x + tau * cx + q * (2.0 * w.x * ws - w2 * s.x);
  double y = s.y + tau * cy + q * (2.0 * w.y * ws - w2 * s.y);
  double z = s.z + tau * cz + q * (2.0 * w.z * ws - w2 * s.z);
  s.x = x * inv; s.y = y * inv; s.z = z * inv;
}

// omega_i = (mu_s mu_B H + sum_j J_ij s_j) / hbar.
__device__ __forceinline__ double3 omega_of(const SlDev& d, int i) {
  double hx = d.zee[0], hy = d.zee[1], hz = d.zee[2];
  int ne = d.exn[i];
  const int* jj = d.exj + (size_t)i * d.max_ex;
  const double* JJ = d.exJ + (size_t)i * d.max_ex;
  for (int k = 0; k < ne; ++k) {
    double J = JJ[k];
    double4_32a sj = d.s[jj[k]];
    hx = fma(J, sj.x, hx);
    hy = fma(J, sj.y, hy);
    hz = fma(J, sj.z, hz);
  }
  const double ih = 1.0 / SL_HBAR;
  return make_double3(hx * ih, hy * ih, hz * ih);
}

__device__ __forceinline__ void update_spin(const SlDev& d, int i, double tau, int subpass, long long step) {
  double3 w = omega_of(d, i);
  double4_32a s = d.s[i];
  if (d.lambda != 0.0 || d.temperature != 0.0) {
    // Eq. sLLG as ds/dt = Om x s, Om = (w + eta + lambda s x w) / (1 + lambda^2),
    // eta ~ N(0, 2 D_S / |tau|), D_S = lambda (1 + lambda^2) k_B T / hbar.
    double lam = d.lambda;
    double3 eta = make_double3(0.0, 0.0, 0.0);
    if (d.temperature > 0.0) {
      double3 g = gauss3(d.seed, d.replica, step, subpass, d.perm[i]);
      double DS = lam * (1.0 + lam * lam) * SL_KB * d.temperature / SL_HBAR;
      double sig = sqrt(2.0 * DS / fabs(tau));
      eta = make_double3(sig * g.x, sig * g.y, sig * g.z);
    }
    double sx = s.y * w.z - s.z * w.y;
    double sy = s.z * w.x - s.x * w.z;
    double sz = s.x * w.y - s.y * w.x;
    double inv = 1.0 / (1.0 + lam * lam);
    w = make_double3((w.x + eta.x + lam * sx) * inv, (w.y + eta.y + lam * sy) * inv,
                     (w.z + eta.z + lam * sz) * inv);
  }
  if (d.rotation == SL_ROT_CAYLEY) rotate_cayley(w, tau, s);
  else rotate_exact(w, tau, s);
  d.s[i] = s;
}

// One colour pass: thread = sector of this colour, its spins in order.
__global__ void k_sweep_pass(SlDev d, int colour, int backward, int subpass, double tau) {
  int qi = blockIdx.x * blockDim.x + threadIdx.x;
  if (qi >= d.s8) return;
  int q = colour * d.s8 + qi;
  int a = d.sec_start[q], b = d.sec_start[q + 1];
  long long step = d.ctrl->step;
  if (!backward) {
    for (int i = a; i < b; ++i) update_spin(d, i, tau, subpass, step);
  } else {
    for (int i = b - 1; i >= a; --i) update_spin(d, i, tau, subpass, step);
  }
}

__global__ void k_kick(SlDev d, double h) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.n) return;
  double c = h * d.acc;
  double4_32a v = d.v[k], F = d.F[k];
  v.x = fma(c, F.x, v.x); v.y = fma(c, F.y, v.y); v.z = fma(c, F.z, v.z);
  d.v[k] = v;
}

// r += dt v and the largest displacement since the last rebuild.
__global__ void k_drift(SlDev d) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  double m = 0.0;
  if (k < d.n) {
    double4_32a r = d.r[k], v = d.v[k], b = d.rb[k];
    r.x = fma(d.dt, v.x, r.x); r.y = fma(d.dt, v.y, r.y); r.z = fma(d.dt, v.z, r.z);
    d.r[k] = r;
    double x = r.x - b.x, y = r.y - b.y, z = r.z - b.z;
    m = x * x + y * y + z * z;
    if (!(m == m) || !(fabs(r.x) + fabs(r.y) + fabs(r.z) < 1e300)) sl_set_error(d.ctrl, SL_ERR_NONFINITE);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0)
    atomicMax(&d.ctrl->maxdisp2_bits, (unsigned long long)__double_as_longlong(m));
}

// Decide whether this step re-sectors (displacement trigger or schedule).
__global__ void k_decide(SlDev d) {
  SlCtrl* c = d.ctrl;
  double md2 = __longlong_as_double((long long)c->maxdisp2_bits);
  int need;
  if (d.rebuild_every > 0) {
    need = ((c->step + 1) % d.rebuild_every) == 0;
    if (!need && md2 > d.half_skin2) sl_set_error(c, SL_ERR_SKIN);
  } else {
    need = md2 > d.half_skin2;
  }
  c->need_rebuild = need;
  c->maxdisp2_bits = 0ull;
}

// Exchange table at the current positions (recomputed after every drift,
// Sec. 3): J_ij and J'_ij e_ij (e_ij = (r_j - r_i)/r_ij), zero beyond ex_rc.
__global__ void k_jtable(SlDev d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  double4_32a ri = d.r[i];
  int ne = d.exn[i];
  size_t base = (size_t)i * d.max_ex;
  double id2 = 1.0 / (d.ex_delta * d.ex_delta);
  for (int k = 0; k < ne; ++k) {
    int j = d.exj[base + k];
    double3 dd = sl_min_image(d, ri, d.r[j]);
    double r2 = dd.x * dd.x + dd.y * dd.y + dd.z * dd.z;
    double J = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    if (r2 < d.ex_rc2) {
      double x = r2 * id2;
      double e = exp(-x);
      J = 4.0 * d.ex_alpha * x * (1.0 - d.ex_gamma * x) * e;
      // J'(r)/r = 8 alpha / delta^2 e^{-x} (1 - 2 g x - x + g x^2)
      double dJr = 8.0 * d.ex_alpha * id2 * e * (1.0 - 2.0 * d.ex_gamma * x - x + d.ex_gamma * x * x);
      gx = dJr * dd.x; gy = dJr * dd.y; gz = dJr * dd.z;
    }
    d.exJ[base + k] = J;
    d.exG[base + k] = make_double4_32a(gx, gy, gz, J);
  }
}

// F_i = sum_j V'(r) e_ij - sum_j J'_ij (s_i.s_j) e_ij, then optionally
// v += (dt/2) F / m (the closing half-kick).
__global__ void k_force(SlDev d, int kick) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  double4_32a ri = d.r[i];
  double fx = 0.0, fy = 0.0, fz = 0.0;
  int nm = d.mn[i];
  double c2 = 2.0 * d.m_alpha * d.m_D0;
  for (int k = 0; k < nm; ++k) {
    int j = d.mj[(size_t)k * d.n + i];
    double3 dd = sl_min_image(d, ri, d.r[j]);
    double r2 = dd.x * dd.x + dd.y * dd.y + dd.z * dd.z;
    if (r2 < d.m_rc2) {
      double rinv = rsqrt(r2);
      double r = r2 * rinv;
      double e = exp(-d.m_alpha * (r - d.m_r0));
      double c = c2 * e * (1.0 - e) * rinv;   // V'(r)/r
      fx = fma(c, dd.x, fx); fy = fma(c, dd.y, fy); fz = fma(c, dd.z, fz);
    }
  }
  double4_32a si = d.s[i];
  int ne = d.exn[i];
  size_t base = (size_t)i * d.max_ex;
  for (int k = 0; k < ne; ++k) {
    double4_32a g = d.exG[base + k];
    double4_32a sj = d.s[d.exj[base + k]];
    double sij = si.x * sj.x + si.y * sj.y + si.z * sj.z;
    fx = fma(-sij, g.x, fx); fy = fma(-sij, g.y, fy); fz = fma(-sij, g.z, fz);
  }
  d.F[i] = make_double4_32a(fx, fy, fz, 0.0);
  if (kick) {
    double c = 0.5 * d.dt * d.acc;
    double4_32a v = d.v[i];
    v.x = fma(c, fx, v.x); v.y = fma(c, fy, v.y); v.z = fma(c, fz, v.z);
    d.v[i] = v;
  }
}

__global__ void k_end_step(SlDev d) { d.ctrl->step += 1; }

void launch_half_op(const SlDev& d, cudaStream_t st, double h, int subpass0) {
  int g = grid_for(d.s8);
  double tau = 0.5 * h;
  for (int c = 0; c < 8; ++c) k_sweep_pass<<<g, SL_BLOCK, 0, st>>>(d, c, 0, subpass0, tau);
  for (int c = 7; c >= 0; --c) k_sweep_pass<<<g, SL_BLOCK, 0, st>>>(d, c, 1, subpass0 + 1, tau);
}

}  // namespace

// Exchange table and forces at the current state (after init/rebuild/set_state).
int sl_launch_pairs_and_forces(const SlDev& d, cudaStream_t st, int kick) {
  int gn = grid_for(d.n);
  k_jtable<<<gn, SL_BLOCK, 0, st>>>(d);
  k_force<<<gn, SL_BLOCK, 0, st>>>(d, kick);
  return cudaPeekAtLastError() == cudaSuccess ? SL_OK : SL_ERR_CUDA;
}

int sl_launch_step(const SlDev& d, cudaStream_t st, SlPhaseMark mark, void* user, int* kernels) {
  int gn = grid_for(d.n);
  const int lat = !d.fix_lattice;
  int nk = 0;
  auto phase = [&](int ph, int end) { if (mark) mark(user, ph, end); };
  if (lat) {
    phase(SL_PHASE_KICK, 0);
    k_kick<<<gn, SL_BLOCK, 0, st>>>(d, 0.5 * d.dt);
    phase(SL_PHASE_KICK, 1);
    nk += 1;
  }
  phase(SL_PHASE_SPIN1, 0);
  launch_half_op(d, st, 0.5 * d.dt, 0);
  phase(SL_PHASE_SPIN1, 1);
  nk += 16;
  if (lat) {
    phase(SL_PHASE_DRIFT, 0);
    k_drift<<<gn, SL_BLOCK, 0, st>>>(d);
    k_decide<<<1, 1, 0, st>>>(d);
    int e = sl_launch_rebuild(d, st);
    if (e) return e;
    phase(SL_PHASE_DRIFT, 1);
    phase(SL_PHASE_JTABLE, 0);
    k_jtable<<<gn, SL_BLOCK, 0, st>>>(d);
    phase(SL_PHASE_JTABLE, 1);
    nk += 2 + SL_REBUILD_KERNELS + 1;
  }
  phase(SL_PHASE_SPIN2, 0);
  launch_half_op(d, st, 0.5 * d.dt, 2);
  phase(SL_PHASE_SPIN2, 1);
  nk += 16;
  if (lat) {
    phase(SL_PHASE_FORCE, 0);
    k_force<<<gn, SL_BLOCK, 0, st>>>(d, 1);
    phase(SL_PHASE_FORCE, 1);
    nk += 1;
  }
  k_end_step<<<1, 1, 0, st>>>(d);
  nk += 1;
  if (kernels) *kernels = nk;
  return cudaPeekAtLastError() == cudaSuccess ? SL_OK : SL_ERR_CUDA;
}

// omega of every atom in caller order (device out [n][3]).
namespace {
__global__ void k_omega_all(SlDev d, double* out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.n) return;
  double3 w = omega_of(d, k);
  int id = d.perm[k];
  out[3 * (size_t)id] = w.x; out[3 * (size_t)id + 1] = w.y; out[3 * (size_t)id + 2] = w.z;
}
}  // namespace

int sl_launch_omega_all(const SlDev& d, double* out, cudaStream_t st) {
  k_omega_all<<<grid_for(d.n), SL_BLOCK, 0, st>>>(d, out);
  return cudaPeekAtLastError() == cudaSuccess ? SL_OK : SL_ERR_CUDA;
}
