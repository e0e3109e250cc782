// Pyramidal Lucas-Kanade optical flow on the device (sim_flow_*): the flow
// the paper's sparse and difference simulators take between consecutive
// frames (Sec. III-B, Sec. IV-A: "Sparse int. w. LK", "Difference int. w.
// LK"), computed here instead of on the host so that frames go straight from
// the flow into the simulator.
//
// Lucas and Kanade take a pixel's flow as the least-squares solution of the
// linearised brightness-constancy equations Ix u + Iy v + It = 0 over a
// window, iterated with the second frame resampled at the current estimate,
// coarse to fine over image pyramids.  Arithmetic (all integer up to the
// 2 x 2 solve, which runs in IEEE double with every operation rounded
// explicitly, so the flow is the same on every run and device):
//   - level 0: 8-bit luma (BT.601 for RGB) times 16; level l+1: 2 x 2 box
//     average of level l, rounded half up, size ((W+1)/2, (H+1)/2), reads
//     clamped;
//   - gradients of the first frame, twice the central difference, reads
//     clamped; window: the (2r+1)^2 pixels p + (i, j) with each coordinate
//     clamped to the image;
//   - G = sums of Ix Ix, Ix Iy, Iy Iy over the window (64-bit); a pixel is
//     tracked when the smaller eigenvalue of G per window pixel is at least
//     min_eig (and det G > 0), else it keeps its guess;
//   - per iteration: It(q) = J(q + g + v) - I(q) with J sampled by the
//     clamped bilinear of the simulator (Q16 position, 12-bit fractions,
//     blends rounded half up); the update -2 G^-1 b, b = sums of (Ix It,
//     Iy It), as each numerator times -2^17 / det G (one division per pixel
//     and level), rounded to Q16; v is clamped to +-1024 px;
//   - the guess of a level-l pixel is twice the flow of its parent
//     (x / 2, y / 2) at level l + 1; the level-0 flow, Q16 px, is written
//     as float pixels.
//
// Kernels: k_lk_base (luma x 16 of both frames), k_lk_down (one pyramid
// level of both frames), k_lk_level (one level's flow: a 32 x 8 block stages
// the gradients and values of its window region in shared memory, one thread
// per pixel).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <new>

#include "../../include/evsim.h"
#include "internal.h"

namespace {

constexpr int LBX = 32, LBY = 8;  // pixels per block of k_lk_level
constexpr int LMAXR = 7;          // largest window radius
constexpr int LMAXL = 8;          // largest number of pyramid levels
constexpr int TXW = LBX + 2 * LMAXR, TYH = LBY + 2 * LMAXR;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

__device__ __forceinline__ int luma_at(const unsigned char* f, long long pitch, int ch, int x,
                                       int y) {
  const unsigned char* q = f + (long long)y * pitch + (long long)x * ch;
  if (ch == 1) return q[0];
  return (77 * q[0] + 150 * q[1] + 29 * q[2] + 128) >> 8;
}

__global__ void k_lk_base(const unsigned char* f0, long long p0, const unsigned char* f1,
                          long long p1, int ch, int W, int H, short* I, short* J) {
  const long long P = (long long)W * H;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(i / W), x = (int)(i - (long long)y * W);
    I[i] = (short)(16 * luma_at(f0, p0, ch, x, y));
    J[i] = (short)(16 * luma_at(f1, p1, ch, x, y));
  }
}

__global__ void k_lk_down(const short* Is, const short* Js, int ws, int hs, short* Id, short* Jd,
                          int wd, int hd) {
  const long long P = (long long)wd * hd;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(i / wd), x = (int)(i - (long long)y * wd);
    const int x0 = 2 * x, x1 = min(2 * x + 1, ws - 1);
    const int y0 = 2 * y, y1 = min(2 * y + 1, hs - 1);
    const long long r0 = (long long)y0 * ws, r1 = (long long)y1 * ws;
    const int si = Is[r0 + x0] + Is[r0 + x1] + Is[r1 + x0] + Is[r1 + x1];
    const int sj = Js[r0 + x0] + Js[r0 + x1] + Js[r1 + x0] + Js[r1 + x1];
    Id[i] = (short)((si + 2) >> 2);
    Jd[i] = (short)((sj + 2) >> 2);
  }
}

// Clamped bilinear sample of a Q4 level image at a Q16 position (blends
// a + floor(((b - a) f + 2048) / 4096), evaluated as one shifted sum).
__device__ __forceinline__ int lk_sample(const short* P, int w, int h, long long px,
                                         long long py) {
  px = px < 0 ? 0 : (px > (long long)(w - 1) << 16 ? (long long)(w - 1) << 16 : px);
  py = py < 0 ? 0 : (py > (long long)(h - 1) << 16 ? (long long)(h - 1) << 16 : py);
  const int ix = (int)(px >> 16), iy = (int)(py >> 16);
  const int fx = (int)((px & 0xFFFF) >> 4), fy = (int)((py & 0xFFFF) >> 4);
  const int x1 = min(ix + 1, w - 1), y1 = min(iy + 1, h - 1);
  const long long r0 = (long long)iy * w, r1 = (long long)y1 * w;
  const int l00 = __ldg(P + r0 + ix), l01 = __ldg(P + r0 + x1);
  const int l10 = __ldg(P + r1 + ix), l11 = __ldg(P + r1 + x1);
  const int top = (l00 * (4096 - fx) + l01 * fx + 2048) >> 12;
  const int bot = (l10 * (4096 - fx) + l11 * fx + 2048) >> 12;
  return (top * (4096 - fy) + bot * fy + 2048) >> 12;
}

struct LevelArg {
  const short* I;
  const short* J;
  int w, h;
  const int* Dup;   // flow of level l + 1 (2 ints per pixel, Q16), null at the top
  int wu;           // its width
  int* D;           // flow of this level
  float* out;       // level 0: the float output (else null)
  int r, iters;
  double min_eig, area;
};

__global__ void __launch_bounds__(LBX * LBY) k_lk_level(LevelArg a) {
  __shared__ short sIx[TYH][TXW], sIy[TYH][TXW], sI[TYH][TXW];
  const int r = a.r, w = a.w, h = a.h;
  const int bx0 = blockIdx.x * LBX, by0 = blockIdx.y * LBY;
  const int tw = LBX + 2 * r, th = LBY + 2 * r;
  // stage the window region: each element is the clamped pixel's value and
  // gradients (window coordinates are clamped before the gradient is taken)
  for (int e = threadIdx.x; e < tw * th; e += LBX * LBY) {
    const int ty = e / tw, tx = e - ty * tw;
    const int qx = clampi(bx0 - r + tx, 0, w - 1), qy = clampi(by0 - r + ty, 0, h - 1);
    const long long row = (long long)qy * w;
    const int xm = max(qx - 1, 0), xp = min(qx + 1, w - 1);
    const int ym = max(qy - 1, 0), yp = min(qy + 1, h - 1);
    sI[ty][tx] = a.I[row + qx];
    sIx[ty][tx] = (short)(a.I[row + xp] - a.I[row + xm]);
    sIy[ty][tx] = (short)(a.I[(long long)yp * w + qx] - a.I[(long long)ym * w + qx]);
  }
  __syncthreads();
  const int lx = threadIdx.x % LBX, ly = threadIdx.x / LBX;
  const int x = bx0 + lx, y = by0 + ly;
  if (x >= w || y >= h) return;
  long long gx = 0, gy = 0;
  if (a.Dup) {
    const long long pp = (long long)(y >> 1) * a.wu + (x >> 1);
    gx = 2LL * a.Dup[2 * pp];
    gy = 2LL * a.Dup[2 * pp + 1];
  }
  long long sxx = 0, sxy = 0, syy = 0;
  for (int j = 0; j <= 2 * r; ++j)
    for (int i = 0; i <= 2 * r; ++i) {
      const long long ix = sIx[ly + j][lx + i], iy = sIy[ly + j][lx + i];
      sxx += ix * ix;
      sxy += ix * iy;
      syy += iy * iy;
    }
  const double A = (double)sxx, B = (double)sxy, Dd = (double)syy;
  const double det = __dsub_rn(__dmul_rn(A, Dd), __dmul_rn(B, B));
  const double tr = __dadd_rn(A, Dd), df = __dsub_rn(A, Dd);
  const double disc = __dsqrt_rn(__dadd_rn(__dmul_rn(df, df), __dmul_rn(__dmul_rn(4.0, B), B)));
  const double lmin = __dmul_rn(__dsub_rn(tr, disc), 0.5);
  const long long lim = 1024LL * 65536;
  long long vx = 0, vy = 0;
  if (__ddiv_rn(lmin, a.area) >= a.min_eig && det > 0.0) {
    const double scale = __ddiv_rn(-131072.0, det);
    for (int k = 0; k < a.iters; ++k) {
      long long bxs = 0, bys = 0;
      for (int j = 0; j <= 2 * r; ++j) {
        const int qy = clampi(y - r + j, 0, h - 1);
        for (int i = 0; i <= 2 * r; ++i) {
          const int qx = clampi(x - r + i, 0, w - 1);
          const int jv = lk_sample(a.J, w, h, ((long long)qx << 16) + gx + vx,
                                   ((long long)qy << 16) + gy + vy);
          const long long it = jv - sI[ly + j][lx + i];
          bxs += sIx[ly + j][lx + i] * it;
          bys += sIy[ly + j][lx + i] * it;
        }
      }
      const double ex = (double)bxs, ey = (double)bys;
      const double nx = __dsub_rn(__dmul_rn(Dd, ex), __dmul_rn(B, ey));
      const double ny = __dsub_rn(__dmul_rn(A, ey), __dmul_rn(B, ex));
      vx += __double2ll_rn(__dmul_rn(nx, scale));
      vy += __double2ll_rn(__dmul_rn(ny, scale));
      vx = vx > lim ? lim : (vx < -lim ? -lim : vx);
      vy = vy > lim ? lim : (vy < -lim ? -lim : vy);
    }
  }
  long long ox = gx + vx, oy = gy + vy;
  ox = ox > lim ? lim : (ox < -lim ? -lim : ox);
  oy = oy > lim ? lim : (oy < -lim ? -lim : oy);
  const long long p = (long long)y * w + x;
  if (a.out) {
    a.out[2 * p] = __int2float_rn((int)ox) * (1.0f / 65536.0f);
    a.out[2 * p + 1] = __int2float_rn((int)oy) * (1.0f / 65536.0f);
  } else {
    a.D[2 * p] = (int)ox;
    a.D[2 * p + 1] = (int)oy;
  }
}

}  // namespace

struct sim_flow_s {
  sim_flow_config cfg{};
  int W = 0, H = 0, L = 1;
  int ws[LMAXL] = {}, hs[LMAXL] = {};
  short* I[LMAXL] = {};
  short* J[LMAXL] = {};
  int* D[LMAXL] = {};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int sms = 1;
};

namespace {

void flow_free(sim_flow_t* f) {
  for (int l = 0; l < LMAXL; ++l) {
    cudaFree(f->I[l]);
    cudaFree(f->J[l]);
    cudaFree(f->D[l]);
  }
  if (f->own_stream && f->stream) cudaStreamDestroy(f->stream);
}

int flow_rc(cudaError_t e) {
  evsim::note_cuda_error(e);
  if (e == cudaErrorMemoryAllocation) return SIM_ERR_OOM;
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver ||
      e == cudaErrorNoKernelImageForDevice)
    return SIM_ERR_NO_DEVICE;
  return SIM_ERR_CUDA;
}

}  // namespace

extern "C" {

int sim_flow_config_default(sim_flow_config* c, int32_t width, int32_t height) {
  if (!c) return SIM_ERR_ARG;
  *c = sim_flow_config{};
  c->width = width;
  c->height = height;
  c->pixel_format = SIM_LUMA8;
  c->levels = 3;
  c->radius = 3;
  c->iterations = 3;
  c->min_eig = 64.0;
  return SIM_OK;
}

int sim_flow_create(const sim_flow_config* cfg, sim_flow_t** out) {
  if (!cfg || !out) return SIM_ERR_ARG;
  const sim_flow_config& c = *cfg;
  if (c.width < 1 || c.height < 1 || c.width > SIM_MAX_DIM || c.height > SIM_MAX_DIM)
    return SIM_ERR_ARG;
  if (c.pixel_format != SIM_LUMA8 && c.pixel_format != SIM_RGB8) return SIM_ERR_ARG;
  if (c.levels < 1 || c.levels > LMAXL || c.radius < 1 || c.radius > LMAXR) return SIM_ERR_ARG;
  if (c.iterations < 1 || c.iterations > 16) return SIM_ERR_ARG;
  if (!(c.min_eig >= 0.0) || c.min_eig > 1e300) return SIM_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return SIM_ERR_NO_DEVICE;
  sim_flow_t* f = new (std::nothrow) sim_flow_t();
  if (!f) return SIM_ERR_OOM;
  f->cfg = c;
  f->W = c.width;
  f->H = c.height;
  f->L = c.levels;
  f->sms = std::max(1, evsim::device_sm_count());
  cudaError_t e = cudaSuccess;
  if (c.cuda_stream) {
    f->stream = (cudaStream_t)c.cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&f->stream, cudaStreamNonBlocking);
    f->own_stream = e == cudaSuccess;
  }
  int w = c.width, h = c.height;
  for (int l = 0; l < f->L && e == cudaSuccess; ++l) {
    f->ws[l] = w;
    f->hs[l] = h;
    const size_t n = (size_t)w * h;
    e = cudaMalloc(&f->I[l], n * sizeof(short));
    if (e == cudaSuccess) e = cudaMalloc(&f->J[l], n * sizeof(short));
    if (e == cudaSuccess && l > 0) e = cudaMalloc(&f->D[l], 2 * n * sizeof(int));
    w = (w + 1) / 2;
    h = (h + 1) / 2;
  }
  if (e != cudaSuccess) {
    const int rc = flow_rc(e);
    flow_free(f);
    delete f;
    return rc;
  }
  *out = f;
  return SIM_OK;
}

int sim_flow_compute(sim_flow_t* f, const void* prev, int64_t prev_pitch, const void* cur,
                     int64_t cur_pitch, float* flow) {
  if (!f || !prev || !cur || !flow) return SIM_ERR_ARG;
  const long long row = (long long)f->W * f->cfg.pixel_format;
  if (prev_pitch < row || cur_pitch < row) return SIM_ERR_ARG;
  if (((uintptr_t)flow & 7) != 0) return SIM_ERR_ARG;
  cudaStream_t st = f->stream;
  auto grid_of = [&](long long n) {
    return (int)std::max(1LL, std::min<long long>((n + 255) / 256, (long long)f->sms * 8));
  };
  k_lk_base<<<grid_of((long long)f->W * f->H), 256, 0, st>>>(
      (const unsigned char*)prev, prev_pitch, (const unsigned char*)cur, cur_pitch,
      f->cfg.pixel_format, f->W, f->H, f->I[0], f->J[0]);
  cudaError_t e = cudaGetLastError();
  for (int l = 1; l < f->L && e == cudaSuccess; ++l) {
    k_lk_down<<<grid_of((long long)f->ws[l] * f->hs[l]), 256, 0, st>>>(
        f->I[l - 1], f->J[l - 1], f->ws[l - 1], f->hs[l - 1], f->I[l], f->J[l], f->ws[l],
        f->hs[l]);
    e = cudaGetLastError();
  }
  const int r = f->cfg.radius;
  for (int l = f->L - 1; l >= 0 && e == cudaSuccess; --l) {
    LevelArg a;
    a.I = f->I[l];
    a.J = f->J[l];
    a.w = f->ws[l];
    a.h = f->hs[l];
    a.Dup = l + 1 < f->L ? f->D[l + 1] : nullptr;
    a.wu = l + 1 < f->L ? f->ws[l + 1] : 0;
    a.D = f->D[l];
    a.out = l == 0 ? flow : nullptr;
    a.r = r;
    a.iters = f->cfg.iterations;
    a.min_eig = f->cfg.min_eig;
    a.area = (double)((2 * r + 1) * (2 * r + 1));
    const dim3 grid((a.w + LBX - 1) / LBX, (a.h + LBY - 1) / LBY);
    k_lk_level<<<grid, LBX * LBY, 0, st>>>(a);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? SIM_OK : flow_rc(e);
}

int sim_flow_destroy(sim_flow_t* f) {
  if (!f) return SIM_ERR_ARG;
  cudaStreamSynchronize(f->stream);
  flow_free(f);
  delete f;
  return SIM_OK;
}

}  // extern "C"
