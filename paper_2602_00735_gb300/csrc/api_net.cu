// Host side of the learned coarse correction: the network's device state
// (FP32 master parameters, Adam moments, BF16 weight tiles, activations),
// its forward and backward passes as sequences of the kernels in cnn.cu,
// training on residual/error pairs, and the FGMRES with the learned stage.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "net_internal.h"

using rp::c128;
using rp::dalloc;
using rp::dfree;

namespace {

constexpr int kL = 6;
int cr(int i) { return (i == 0 || i == kL) ? 2 : 32; }    // real channels
int cp(int i) { return (i == 0 || i == kL) ? 16 : 32; }   // padded channels

}  // namespace

struct ras_pml_net {
  int dev = 0;
  cudaStream_t st = nullptr;
  int Nc = 0, cap = 0;
  long long npix = 0;
  int nparam = 0;
  int w_off[kL] = {}, b_off[kL] = {};
  float *params = nullptr, *grads = nullptr, *m1 = nullptr, *m2 = nullptr;
  void* wf[kL] = {};        // forward B tiles (BF16)
  void* wd[kL] = {};        // data-gradient B tiles (BF16), layers 1..5
  float* bpad[kL] = {};     // biases padded to the layer's output channels
  void* act[kL] = {};       // layer inputs (BF16 NHWC): act[0] 16 channels, others 32
  float* out = nullptr;     // last layer output (FP32 NHWC, 16 channels)
  void *g0 = nullptr, *g1 = nullptr;   // gradient ping-pong (BF16 NHWC, 32 channels)
  float *xin = nullptr, *tgt = nullptr;   // NCHW FP32 staging (2 channels)
  float* part = nullptr;    // per-block partial weight gradients
  int part_blocks = 0;
  double* lossbuf = nullptr;
  double* rpart = nullptr;  // partial sums of the restriction
  double* sdev = nullptr;   // ||restrict(r1)|| of the last correction
  rp::DevStatus* status = nullptr;
  bool tiles_ok = false;
  long long adam_t = 0;
  double gamma = 1.0;       // output scale of the correction
};

namespace {

int net_tiles(ras_pml_net* n, cudaStream_t st) {
  if (n->tiles_ok) return RASPML_OK;
  for (int l = 0; l < kL; ++l) {
    RP_CUDA(rp::launch_prep_weights(n->params + n->w_off[l], l, 0, n->wf[l], st));
    if (l > 0) RP_CUDA(rp::launch_prep_weights(n->params + n->w_off[l], l, 1, n->wd[l], st));
    RP_CUDA(rp::launch_pad_bias(n->params + n->b_off[l], l, n->bpad[l], st));
  }
  n->tiles_ok = true;
  return RASPML_OK;
}

// forward over nimg images already in act[0]; output in n->out
int net_forward_dev(ras_pml_net* n, int nimg, cudaStream_t st) {
  int s = net_tiles(n, st);
  if (s != RASPML_OK) return s;
  for (int l = 0; l < kL; ++l) {
    const bool last = l == kL - 1;
    RP_CUDA(rp::launch_conv(cp(l), cp(l + 1), n->act[l], n->wf[l], n->bpad[l], nullptr, last ? 0 : 1, n->Nc, n->Nc,
                            nimg, last ? nullptr : n->act[l + 1], last ? n->out : nullptr, n->status, st));
  }
  return RASPML_OK;
}

// gradients of the mean loss over nimg images whose forward pass has run;
// the output gradient is in g0 (16 channels)
int net_backward_dev(ras_pml_net* n, int nimg) {
  const int need = rp::wgrad_blocks(n->Nc, n->cap) * (32 * 32 * 9 + 32);
  if (n->part_blocks < need) {
    dfree(n->part);
    int s = dalloc(&n->part, (size_t)need);
    if (s != RASPML_OK) return s;
    n->part_blocks = need;
  }
  void* g = n->g0;
  void* gn = n->g1;
  for (int l = kL - 1; l >= 0; --l) {
    RP_CUDA(rp::launch_wgrad(l, n->act[l], g, n->Nc, n->Nc, nimg, n->part, n->grads + n->w_off[l], n->st));
    if (l > 0) {
      // gradient of layer l's input, masked by the ReLU that produced it
      RP_CUDA(rp::launch_conv(cp(l + 1), cp(l), g, n->wd[l], nullptr, n->act[l], 0, n->Nc, n->Nc, nimg, gn, nullptr,
                              n->status, n->st));
      void* t = g;
      g = gn;
      gn = t;
    }
  }
  return RASPML_OK;
}

// loss and gradients for x (NCHW FP32, device) against t; loss on the host
int net_loss_grad_dev(ras_pml_net* n, const float* x, const float* t, int nimg, double* loss) {
  RP_CUDA(rp::launch_to_nhwc16(x, n->npix, nimg, n->act[0], n->st));
  int s = net_forward_dev(n, nimg, n->st);
  if (s != RASPML_OK) return s;
  int nparts = 0;
  RP_CUDA(rp::launch_loss_grad(n->out, t, n->npix, nimg, n->g0, n->lossbuf, &nparts, n->st));
  s = net_backward_dev(n, nimg);
  if (s != RASPML_OK) return s;
  if (loss) {
    std::vector<double> lp(nparts);
    RP_CUDA(cudaMemcpyAsync(lp.data(), n->lossbuf, sizeof(double) * nparts, cudaMemcpyDeviceToHost, n->st));
    RP_CUDA(cudaStreamSynchronize(n->st));
    double sum = 0.0;
    for (double v : lp) sum += v;
    *loss = sum;
  }
  return RASPML_OK;
}

}  // namespace

namespace rp {

int net_grid(const ras_pml_net* n) { return n->Nc; }

int net_correct(ras_pml_net* n, const c128* r1, c128* z, int nx, int ny, const KState* kst, cudaStream_t st) {
  RP_CUDA(launch_restrict(r1, nx, ny, n->Nc, n->xin, n->rpart, kst, st));
  RP_CUDA(launch_normalise(n->xin, n->Nc, n->rpart, n->sdev, kst, st));
  RP_CUDA(launch_to_nhwc16(n->xin, n->npix, 1, n->act[0], st));
  int s = net_forward_dev(n, 1, st);
  if (s != RASPML_OK) return s;
  RP_CUDA(launch_prolong_add(n->out, n->Nc, nx, ny, n->sdev, n->gamma, z, kst, st));
  return RASPML_OK;
}

}  // namespace rp

namespace {

// splitmix64 + Box-Muller: He-normal initial weights (host side)
uint64_t splitmix(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" {

void ras_pml_net_destroy(ras_pml_net* n) {
  if (!n) return;
  cudaSetDevice(n->dev);
  if (n->st) cudaStreamSynchronize(n->st);
  dfree(n->params); dfree(n->grads); dfree(n->m1); dfree(n->m2);
  for (int l = 0; l < kL; ++l) {
    dfree(n->wf[l]); dfree(n->wd[l]); dfree(n->bpad[l]); dfree(n->act[l]);
  }
  dfree(n->out); dfree(n->g0); dfree(n->g1); dfree(n->xin); dfree(n->tgt); dfree(n->part); dfree(n->lossbuf);
  dfree(n->status); dfree(n->rpart); dfree(n->sdev);
  delete n;
}

int ras_pml_net_create(int Nc, int cap, uint64_t seed, void* stream, ras_pml_net** out) {
  if (!out || Nc < 8 || Nc > 4096 || cap < 1 || cap > 4096) return RASPML_EBADARG;
  *out = nullptr;
  ras_pml_net* n = new ras_pml_net();
  cudaGetDevice(&n->dev);
  n->st = (cudaStream_t)stream;
  n->Nc = Nc;
  n->cap = cap;
  n->npix = (long long)Nc * Nc;
  int off = 0;
  for (int l = 0; l < kL; ++l) {
    n->w_off[l] = off;
    off += cr(l + 1) * cr(l) * 9;
    n->b_off[l] = off;
    off += cr(l + 1);
  }
  n->nparam = off;
  int s;
  const long long np = n->npix * cap;
#define NA(ptr, cnt) \
  if ((s = dalloc(&(ptr), (cnt))) != RASPML_OK) { ras_pml_net_destroy(n); return s; }
  NA(n->params, (size_t)off);
  NA(n->grads, (size_t)off);
  NA(n->m1, (size_t)off);
  NA(n->m2, (size_t)off);
  for (int l = 0; l < kL; ++l) {
    uint16_t* t = nullptr;
    NA(t, (size_t)9 * cp(l) * cp(l + 1));
    n->wf[l] = t;
    if (l > 0) {
      uint16_t* t2 = nullptr;
      NA(t2, (size_t)9 * cp(l) * cp(l + 1));
      n->wd[l] = t2;
    }
    NA(n->bpad[l], (size_t)cp(l + 1));
    uint16_t* a = nullptr;
    NA(a, (size_t)np * cp(l));
    n->act[l] = a;
  }
  NA(n->out, (size_t)np * 16);
  uint16_t *g0 = nullptr, *g1 = nullptr;
  NA(g0, (size_t)np * 32);
  NA(g1, (size_t)np * 32);
  n->g0 = g0;
  n->g1 = g1;
  NA(n->xin, (size_t)np * 2);
  NA(n->tgt, (size_t)np * 2);
  NA(n->lossbuf, (size_t)((n->npix + 255) / 256 * cap));
  NA(n->status, (size_t)1);
  NA(n->rpart, (size_t)rp::restrict_blocks(Nc));
  NA(n->sdev, (size_t)1);
#undef NA
  // He-normal weights, zero biases
  std::vector<float> p(off, 0.f);
  uint64_t state = seed;
  for (int l = 0; l < kL; ++l) {
    const double sd = std::sqrt(2.0 / (9.0 * cr(l)));
    for (int i = 0; i < cr(l + 1) * cr(l) * 9; ++i) {
      const double u1 = ((splitmix(state) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
      const double u2 = ((splitmix(state) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
      p[n->w_off[l] + i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
    }
  }
  cudaError_t e = cudaMemcpyAsync(n->params, p.data(), sizeof(float) * off, cudaMemcpyHostToDevice, n->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->m1, 0, sizeof(float) * off, n->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->m2, 0, sizeof(float) * off, n->st);
  rp::DevStatus s0{-1, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(n->status, &s0, sizeof(s0), cudaMemcpyHostToDevice, n->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->st);
  if (e != cudaSuccess) {
    ras_pml_net_destroy(n);
    return RASPML_ECUDA;
  }
  *out = n;
  return RASPML_OK;
}

int ras_pml_net_param_count(const ras_pml_net* n) { return n ? n->nparam : -1; }

int ras_pml_net_set_params(ras_pml_net* n, const float* host, int count) {
  if (!n || !host || count != n->nparam) return RASPML_EBADARG;
  cudaSetDevice(n->dev);
  RP_CUDA(cudaMemcpyAsync(n->params, host, sizeof(float) * count, cudaMemcpyHostToDevice, n->st));
  RP_CUDA(cudaMemsetAsync(n->m1, 0, sizeof(float) * count, n->st));
  RP_CUDA(cudaMemsetAsync(n->m2, 0, sizeof(float) * count, n->st));
  RP_CUDA(cudaStreamSynchronize(n->st));
  n->adam_t = 0;
  n->tiles_ok = false;
  return RASPML_OK;
}

int ras_pml_net_get_params(const ras_pml_net* n, float* host, int count) {
  if (!n || !host || count != n->nparam) return RASPML_EBADARG;
  cudaSetDevice(n->dev);
  RP_CUDA(cudaMemcpyAsync(host, n->params, sizeof(float) * count, cudaMemcpyDeviceToHost, n->st));
  RP_CUDA(cudaStreamSynchronize(n->st));
  return RASPML_OK;
}

int ras_pml_net_forward(ras_pml_net* n, const float* x_dev, float* y_dev, int nimg) {
  if (!n || !x_dev || !y_dev || nimg < 1 || nimg > n->cap) return RASPML_EBADARG;
  cudaSetDevice(n->dev);
  RP_CUDA(rp::launch_to_nhwc16(x_dev, n->npix, nimg, n->act[0], n->st));
  int s = net_forward_dev(n, nimg, n->st);
  if (s != RASPML_OK) return s;
  RP_CUDA(rp::launch_from_nhwc16(n->out, n->npix, nimg, y_dev, n->st));
  rp::DevStatus stt;
  RP_CUDA(cudaMemcpyAsync(&stt, n->status, sizeof(stt), cudaMemcpyDeviceToHost, n->st));
  RP_CUDA(cudaStreamSynchronize(n->st));
  return stt.timeout ? RASPML_ETIMEOUT : RASPML_OK;
}

int ras_pml_net_loss_grad(ras_pml_net* n, const float* x_dev, const float* t_dev, int nimg, double* loss_host,
                          float* grad_host) {
  if (!n || !x_dev || !t_dev || nimg < 1 || nimg > n->cap || !loss_host) return RASPML_EBADARG;
  cudaSetDevice(n->dev);
  int s = net_loss_grad_dev(n, x_dev, t_dev, nimg, loss_host);
  if (s != RASPML_OK) return s;
  if (grad_host) {
    RP_CUDA(cudaMemcpyAsync(grad_host, n->grads, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost, n->st));
  }
  rp::DevStatus stt;
  RP_CUDA(cudaMemcpyAsync(&stt, n->status, sizeof(stt), cudaMemcpyDeviceToHost, n->st));
  RP_CUDA(cudaStreamSynchronize(n->st));
  return stt.timeout ? RASPML_ETIMEOUT : RASPML_OK;
}

int ras_pml_net_adam_step(ras_pml_net* n, float lr) {
  if (!n || !(lr > 0.f)) return RASPML_EBADARG;
  cudaSetDevice(n->dev);
  n->adam_t += 1;
  RP_CUDA(rp::launch_adam(n->params, n->grads, n->m1, n->m2, n->nparam, lr, n->adam_t, n->st));
  n->tiles_ok = false;
  return RASPML_OK;
}

int ras_pml_net_set_gamma(ras_pml_net* n, double gamma) {
  if (!n || !(gamma > 0.0)) return RASPML_EBADARG;
  n->gamma = gamma;
  return RASPML_OK;
}

double ras_pml_net_get_gamma(const ras_pml_net* n) { return n ? n->gamma : 0.0; }

int ras_pml_net_train(ras_pml_net* n, ras_pml_handle* h, int nrhs, const int32_t* m_list, int nm, int epochs, float lr,
                      uint64_t seed, float* loss_hist, double* gamma_out) {
  if (!n || !h || nrhs < 1 || !m_list || nm < 1 || epochs < 1 || !(lr > 0.f) || !loss_hist) return RASPML_EBADARG;
  for (int i = 0; i < nm; ++i)
    if (m_list[i] < 1) return RASPML_EBADARG;
  cudaSetDevice(n->dev);
  ras_pml_info_t inf;
  ras_pml_params prm;
  int s = ras_pml_info(h, &inf);
  if (s == RASPML_OK) s = ras_pml_get_params(h, &prm);
  if (s != RASPML_OK) return s;
  const int nx = inf.Mx - 1, ny = inf.My - 1;
  if (n->Nc > nx || n->Nc > ny) return RASPML_EBADARG;
  const long long nn = inf.n;
  const int ns = nrhs * nm;
  const long long img = 2 * n->npix;
  // pairs are generated with the plain method: detach any learned stage
  ras_pml_attach_net(h, nullptr);
  c128 *b = nullptr, *xs = nullptr, *xm = nullptr, *r = nullptr, *e = nullptr, *t = nullptr;
  float *X = nullptr, *T = nullptr;
  std::vector<double> sr(ns), gam(ns);
  cudaError_t ce = cudaSuccess;
  auto cleanup = [&]() {
    dfree(b); dfree(xs); dfree(xm); dfree(r); dfree(e); dfree(t); dfree(X); dfree(T);
  };
#define TA(ptr, cnt) \
  if ((s = dalloc(&(ptr), (cnt))) != RASPML_OK) { cleanup(); return s; }
  TA(b, (size_t)nn);
  TA(xs, (size_t)nn);
  TA(xm, (size_t)nn);
  TA(r, (size_t)nn);
  TA(e, (size_t)nn);
  TA(t, (size_t)nn);
  TA(X, (size_t)ns * img);
  TA(T, (size_t)ns * img);
#undef TA
#define TCHK(call)                                                         \
  do {                                                                     \
    if ((ce = (call)) != cudaSuccess) {                                    \
      std::fprintf(stderr, "raspml: train: %s\n", cudaGetErrorString(ce)); \
      cleanup();                                                           \
      return RASPML_ECUDA;                                                 \
    }                                                                      \
  } while (0)
  uint64_t st = seed;
  auto unif = [&]() { return ((splitmix(st) >> 11) + 0.5) * (1.0 / 9007199254740992.0); };
  const double width = 0.4 * 3.141592653589793 / prm.k;
  for (int k = 0; k < nrhs; ++k) {
    // load vector of 1-8 Gaussian sources at random points of Omega_int
    const int nsrc = 1 + (int)(unif() * 8.0);
    std::vector<double> cen(2 * nsrc), amp(nsrc, 1.0);
    for (int q = 0; q < nsrc; ++q) {
      cen[2 * q] = prm.x0 + unif() * (prm.x1 - prm.x0);
      cen[2 * q + 1] = prm.y0 + unif() * (prm.y1 - prm.y0);
    }
    if ((s = ras_pml_assemble_rhs(h, cen.data(), amp.data(), nsrc, width, (rp_c128*)b)) != RASPML_OK) break;
    TCHK(cudaMemset(xs, 0, sizeof(c128) * nn));
    int it;
    double rel;
    s = helmholtz_solve(h, (rp_c128*)b, (rp_c128*)xs, 1e-9, 2000, 0, &it, &rel);
    if (s < 0) break;
    for (int q = 0; q < nm; ++q) {
      const int i = k * nm + q;
      // x_m after m directions, its residual and error
      TCHK(cudaMemset(xm, 0, sizeof(c128) * nn));
      s = helmholtz_solve(h, (rp_c128*)b, (rp_c128*)xm, 0.0, m_list[q], 0, &it, &rel);
      if (s < 0) break;
      if ((s = ras_pml_matvec(h, (rp_c128*)xm, (rp_c128*)t)) != RASPML_OK) break;
      TCHK(cudaDeviceSynchronize());
      TCHK(rp::launch_csub(b, t, r, nn, n->st));
      TCHK(rp::launch_csub(xs, xm, e, nn, n->st));
      TCHK(rp::launch_restrict(r, nx, ny, n->Nc, X + i * img, n->rpart, nullptr, n->st));
      TCHK(rp::launch_normalise(X + i * img, n->Nc, n->rpart, n->sdev, nullptr, n->st));
      TCHK(cudaMemcpyAsync(&sr[i], n->sdev, sizeof(double), cudaMemcpyDeviceToHost, n->st));
      TCHK(rp::launch_restrict(e, nx, ny, n->Nc, T + i * img, n->rpart, nullptr, n->st));
      std::vector<double> part(rp::restrict_blocks(n->Nc));
      TCHK(cudaMemcpyAsync(part.data(), n->rpart, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, n->st));
      TCHK(cudaStreamSynchronize(n->st));
      const double se = std::sqrt(std::accumulate(part.begin(), part.end(), 0.0));
      gam[i] = sr[i] > 0.0 ? se / sr[i] : 0.0;
    }
    if (s < 0) break;
  }
  if (s < 0) {
    cleanup();
    return s;
  }
  // output scale: the median ratio ||R e|| / ||R r|| over the pairs; the
  // targets become R e * Nc / (gamma ||R r||)
  std::vector<double> gs = gam;
  std::sort(gs.begin(), gs.end());
  const double gamma = gs[ns / 2] > 0.0 ? gs[ns / 2] : 1.0;
  for (int i = 0; i < ns; ++i)
    TCHK(rp::launch_scale_f32(T + i * img, img, sr[i] > 0.0 ? (float)(n->Nc / (gamma * sr[i])) : 0.f, n->st));
  n->gamma = gamma;
  if (gamma_out) *gamma_out = gamma;
  // Adam over shuffled minibatches of up to cap pairs
  std::vector<int> perm(ns);
  std::iota(perm.begin(), perm.end(), 0);
  for (int ep = 0; ep < epochs; ++ep) {
    for (int i = ns - 1; i > 0; --i) std::swap(perm[i], perm[(int)(unif() * (i + 1))]);
    double lsum = 0.0;
    int nb = 0;
    for (int i0 = 0; i0 < ns; i0 += n->cap) {
      const int cnt = std::min(n->cap, ns - i0);
      for (int q = 0; q < cnt; ++q) {
        TCHK(cudaMemcpyAsync(n->xin + q * img, X + perm[i0 + q] * img, sizeof(float) * img, cudaMemcpyDeviceToDevice,
                             n->st));
        TCHK(cudaMemcpyAsync(n->tgt + q * img, T + perm[i0 + q] * img, sizeof(float) * img, cudaMemcpyDeviceToDevice,
                             n->st));
      }
      double L = 0.0;
      if ((s = net_loss_grad_dev(n, n->xin, n->tgt, cnt, &L)) != RASPML_OK) break;
      n->adam_t += 1;
      TCHK(rp::launch_adam(n->params, n->grads, n->m1, n->m2, n->nparam, lr, n->adam_t, n->st));
      n->tiles_ok = false;
      lsum += L;
      ++nb;
    }
    if (s != RASPML_OK) break;
    loss_hist[ep] = (float)(lsum / std::max(nb, 1));
  }
  TCHK(cudaStreamSynchronize(n->st));
#undef TCHK
  cleanup();
  return s;
}

}  // extern "C"
