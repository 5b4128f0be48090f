// Host side of the learned coarse correction: the network's device state
// (FP32 master parameters, Adam moments, BF16 weight tiles, activations),
// its forward and backward passes as sequences of the kernels in cnn.cu,
// training on residual/error pairs, and the FGMRES with the learned stage.
#include <cmath>
#include <cstring>
#include <vector>

#include "host.h"

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
  rp::DevStatus* status = nullptr;
  bool tiles_ok = false;
  long long adam_t = 0;
  double gamma = 1.0;       // output scale of the correction
};

namespace {

int net_tiles(ras_pml_net* n) {
  if (n->tiles_ok) return RASPML_OK;
  for (int l = 0; l < kL; ++l) {
    RP_CUDA(rp::launch_prep_weights(n->params + n->w_off[l], l, 0, n->wf[l], n->st));
    if (l > 0) RP_CUDA(rp::launch_prep_weights(n->params + n->w_off[l], l, 1, n->wd[l], n->st));
    RP_CUDA(rp::launch_pad_bias(n->params + n->b_off[l], l, n->bpad[l], n->st));
  }
  n->tiles_ok = true;
  return RASPML_OK;
}

// forward over nimg images already in act[0]; output in n->out
int net_forward_dev(ras_pml_net* n, int nimg) {
  int s = net_tiles(n);
  if (s != RASPML_OK) return s;
  for (int l = 0; l < kL; ++l) {
    const bool last = l == kL - 1;
    RP_CUDA(rp::launch_conv(cp(l), cp(l + 1), n->act[l], n->wf[l], n->bpad[l], nullptr, last ? 0 : 1, n->Nc, n->Nc,
                            nimg, last ? nullptr : n->act[l + 1], last ? n->out : nullptr, n->status, n->st));
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
  int s = net_forward_dev(n, nimg);
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
  dfree(n->status);
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
  int s = net_forward_dev(n, nimg);
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

}  // extern "C"
