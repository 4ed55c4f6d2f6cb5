// state_energy_noalloc.cu -- kinetic and strain energy of one state of an
// uncracked mesh, computed without allocating any device memory
// (compiled with -fmad=false, like the energy records of the step).
//
// Why this exists: the handle API allocates its device state once, at
// cem_mesh_create.  Some callers cannot allocate at all when they want an
// energy check: a host application that has handed all device memory to its
// own fixed-size arena, or a monitor that samples energies while other
// streams are busy and must not call cudaMalloc / cudaFree (cudaFree
// synchronises the device, which would stall that work).  This entry point
// takes device inputs and a device output from the caller and keeps its only
// scratch -- one (KE, SE) pair per node row -- in a file-scope device array
// that every GPU loading the library holds until the process exits.
//
// The arithmetic is that of the energy record of a step (KE of the given
// velocity with row-sum lumped masses, SE with each element owning A/4 of its
// four ES-FEM edge points, Sec. 2.1): only the partial sums are grouped
// differently (per node row here, per thread block in the step), so the two
// agree to rounding, not bit for bit.
#include <cuda_runtime.h>

#include <climits>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "../../include/cem.h"

namespace {

constexpr int NA_MAX_DEVICES = 64;
constexpr int NA_BLOCK = 256;
constexpr int NA_RED = 1024;

// One (KE, SE) pair per node row: rows = ny + 1 <= CEM_NOALLOC_MAX_NY + 1.
// 16 B per row, 256 KiB + 16 B in all.  Every slot a call reads is written
// earlier in the same call, so nothing here has to start at zero; a call
// with fewer rows simply leaves the previous call's higher rows unread.
static __device__ __align__(256) double g_row_energy[2 * (CEM_NOALLOC_MAX_NY + 1)];

struct NaMesh {
  int nx, ny;
  double hx, hy, rx, ry, q_mass, q_area;  // q_mass = rho*A/4, q_area = A/4
  double D11, D12, D33;
  const unsigned char *act;  // [nx*ny] or nullptr (all active)
  const double *ux, *uy, *vx, *vy;
};

__device__ __forceinline__ bool na_active(const NaMesh &m, int i, int j) {
  if (i < 0 || j < 0 || i >= m.nx || j >= m.ny) return false;
  return m.act == nullptr || m.act[(size_t)j * m.nx + i] != 0;
}

// Own strain of element (i,j) at the midpoint of its local edge k (Eq. 4):
// the Q4 derivatives there are one-sided differences along the edge and the
// mean of the two parallel edges across it.
__device__ void na_own_strain(const NaMesh &m, int i, int j, int k, double eps[3]) {
  const int W = m.nx + 1;
  const size_t n0 = (size_t)j * W + i, n1 = n0 + 1, n2 = n0 + W + 1, n3 = n0 + W;
  const double x0 = m.ux[n0], x1 = m.ux[n1], x2 = m.ux[n2], x3 = m.ux[n3];
  const double y0 = m.uy[n0], y1 = m.uy[n1], y2 = m.uy[n2], y3 = m.uy[n3];
  const double hx2 = 0.5 * m.rx, hy2 = 0.5 * m.ry;
  // differences along x (bottom a, top b) and along y (left c, right e)
  const double au = x1 - x0, bu = x2 - x3, cu = x3 - x0, eu = x2 - x1;
  const double av = y1 - y0, bv = y2 - y3, cv = y3 - y0, ev = y2 - y1;
  switch (k) {
    case 0: eps[0] = m.rx * au; eps[1] = hy2 * (cv + ev); eps[2] = hy2 * (cu + eu) + m.rx * av; break;
    case 1: eps[0] = hx2 * (au + bu); eps[1] = m.ry * ev; eps[2] = m.ry * eu + hx2 * (av + bv); break;
    case 2: eps[0] = m.rx * bu; eps[1] = hy2 * (cv + ev); eps[2] = hy2 * (cu + eu) + m.rx * bv; break;
    default: eps[0] = hx2 * (au + bu); eps[1] = m.ry * cv; eps[2] = m.ry * cu + hx2 * (av + bv); break;
  }
}

__device__ double na_elem_energy(const NaMesh &m, int i, int j) {
  const int di[4] = {0, 1, 0, -1}, dj[4] = {-1, 0, 1, 0};
  double acc = 0.0;
  for (int k = 0; k < 4; ++k) {
    double e[3];
    na_own_strain(m, i, j, k, e);
    // smoothing domain shared with the intact element across edge k
    const int fi = i + di[k], fj = j + dj[k];
    if (na_active(m, fi, fj)) {
      double e2[3];
      na_own_strain(m, fi, fj, (k + 2) & 3, e2);
      for (int c = 0; c < 3; ++c) e[c] = 0.5 * (e[c] + e2[c]);
    }
    const double s0 = m.D11 * e[0] + m.D12 * e[1];
    const double s1 = m.D12 * e[0] + m.D11 * e[1];
    const double s2 = m.D33 * e[2];
    const double d = e[0] * s0 + e[1] * s1 + e[2] * s2;
    acc = acc + 0.5 * (m.q_area * d);
  }
  return acc;
}

__device__ void na_block_sum2(double &a, double &b) {
  __shared__ double wa[32], wb[32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { wa[w] = a; wb[w] = b; }
  __syncthreads();
  if (w == 0) {
    const bool in = lane < (int)(blockDim.x >> 5);
    a = in ? wa[lane] : 0.0;
    b = in ? wb[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
  }
}

// Block j: KE of node row j and SE of element row j (when j < ny), written to
// rows[2j], rows[2j+1].
__global__ void __launch_bounds__(NA_BLOCK) k_row_energy(NaMesh m, double *rows) {
  const int j = blockIdx.x;
  const int W = m.nx + 1;
  double ke = 0.0, se = 0.0;
  for (int i = threadIdx.x; i < W; i += NA_BLOCK) {
    // lumped mass: A/4 * rho from each active element around the node, in the
    // order (i-1,j-1), (i,j-1), (i-1,j), (i,j)
    double mass = 0.0;
    if (na_active(m, i - 1, j - 1)) mass = mass + m.q_mass;
    if (na_active(m, i, j - 1)) mass = mass + m.q_mass;
    if (na_active(m, i - 1, j)) mass = mass + m.q_mass;
    if (na_active(m, i, j)) mass = mass + m.q_mass;
    const size_t N = (size_t)j * W + i;
    const double vx = m.vx[N], vy = m.vy[N];
    ke = ke + 0.5 * (mass * (vx * vx + vy * vy));
    if (i < m.nx && na_active(m, i, j)) se = se + na_elem_energy(m, i, j);
  }
  na_block_sum2(ke, se);
  if (threadIdx.x == 0) {
    rows[2 * j] = ke;
    rows[2 * j + 1] = se;
  }
}

// One block adds the row sums in a fixed order and writes out[0] = KE,
// out[1] = SE.
__global__ void __launch_bounds__(NA_RED) k_rows_total(const double *rows, int n_rows,
                                                       double *out) {
  double ke = 0.0, se = 0.0;
  for (int r = threadIdx.x; r < n_rows; r += NA_RED) {
    ke = ke + rows[2 * r];
    se = se + rows[2 * r + 1];
  }
  na_block_sum2(ke, se);
  if (threadIdx.x == 0) {
    out[0] = ke;
    out[1] = se;
  }
}

// Device address of g_row_energy for each device, looked up once with that
// device current.  In host code the name g_row_energy is only a host-side
// stand-in for the symbol, never a device address.
std::mutex g_na_mutex;
double *g_na_rows[NA_MAX_DEVICES] = {};

cem_status na_fail(char *err, int err_len, cem_status rc, const char *fmt, ...) {
  if (err && err_len > 0) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(err, (size_t)err_len, fmt, ap);
    va_end(ap);
  }
  return rc;
}

// 0 when p is device (or managed) memory usable on device dev.
int na_check_ptr(const void *p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  if (a.type == cudaMemoryTypeManaged) return 0;
  if (a.type != cudaMemoryTypeDevice) return 1;
  return a.device == dev ? 0 : 1;
}

}  // namespace

extern "C" cem_status cem_state_energy_noalloc(int nx, int ny, double hx, double hy,
                                               const unsigned char *elem_active, double E,
                                               double nu, double rho, int plane_strain,
                                               const double *u, const double *v, double *out,
                                               void *cuda_stream, char *err, int err_len) {
  if (err && err_len > 0) err[0] = '\0';
  if (nx < 1 || ny < 1) return na_fail(err, err_len, CEM_ERR_ARG, "nx and ny must be >= 1");
  if (ny > CEM_NOALLOC_MAX_NY)
    return na_fail(err, err_len, CEM_ERR_ARG,
                   "ny = %d exceeds the fixed scratch of this entry point (at most %d element "
                   "rows); use the handle API for larger meshes",
                   ny, CEM_NOALLOC_MAX_NY);
  const long long n_nodes = (long long)(nx + 1LL) * (ny + 1LL);
  if (n_nodes > INT_MAX / 2) return na_fail(err, err_len, CEM_ERR_ARG, "mesh too large");
  if (!(hx > 0) || !(hy > 0)) return na_fail(err, err_len, CEM_ERR_ARG, "hx and hy must be > 0");
  if (!(E > 0) || !(nu > -1.0 && nu < 0.5) || !(rho > 0))
    return na_fail(err, err_len, CEM_ERR_ARG, "bad material (E > 0, -1 < nu < 0.5, rho > 0)");
  if (!u || !v || !out) return na_fail(err, err_len, CEM_ERR_ARG, "u, v and out are required");

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES)
    return na_fail(err, err_len, CEM_ERR_CUDA, "no usable current CUDA device");
  if (na_check_ptr(u, dev) || na_check_ptr(v, dev) || na_check_ptr(out, dev) ||
      (elem_active && na_check_ptr(elem_active, dev)))
    return na_fail(err, err_len, CEM_ERR_ARG,
                   "u, v, out and elem_active must be device memory of the current device");

  double *rows = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    // A cached address that no longer maps to this device's memory (after a
    // cudaDeviceReset, which unloads the module) is looked up again.
    if (g_na_rows[dev] && na_check_ptr(g_na_rows[dev], dev)) {
      cudaGetLastError();
      g_na_rows[dev] = nullptr;
    }
    if (!g_na_rows[dev]) {
      // First call on this device: look up the scratch's device address
      // (this device is current).
      void *p = nullptr;
      cudaError_t ce = cudaGetSymbolAddress(&p, g_row_energy);
      if (ce != cudaSuccess || !p) {
        cudaGetLastError();
        return na_fail(err, err_len, CEM_ERR_CUDA, "cudaGetSymbolAddress: %s",
                       cudaGetErrorString(ce));
      }
      g_na_rows[dev] = static_cast<double *>(p);
    }
    rows = g_na_rows[dev];
  }

  NaMesh m;
  m.nx = nx;
  m.ny = ny;
  m.hx = hx;
  m.hy = hy;
  m.rx = 1.0 / hx;
  m.ry = 1.0 / hy;
  const double A = hx * hy;
  m.q_mass = rho * A * 0.25;
  m.q_area = A * 0.25;
  if (plane_strain) {
    const double c = E / ((1.0 + nu) * (1.0 - 2.0 * nu));
    m.D11 = c * (1.0 - nu);
    m.D12 = c * nu;
    m.D33 = c * (1.0 - 2.0 * nu) * 0.5;
  } else {
    const double c = E / (1.0 - nu * nu);
    m.D11 = c;
    m.D12 = c * nu;
    m.D33 = c * (1.0 - nu) * 0.5;
  }
  m.act = elem_active;
  m.ux = u;
  m.uy = u + n_nodes;
  m.vx = v;
  m.vy = v + n_nodes;

  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  k_row_energy<<<ny + 1, NA_BLOCK, 0, st>>>(m, rows);
  cudaError_t ce = cudaGetLastError();
  if (ce == cudaSuccess) {
    k_rows_total<<<1, NA_RED, 0, st>>>(rows, ny + 1, out);
    ce = cudaGetLastError();
  }
  if (ce != cudaSuccess)
    return na_fail(err, err_len, CEM_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(ce));
  return CEM_OK;
}
