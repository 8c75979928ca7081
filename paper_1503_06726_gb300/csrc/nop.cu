// nop.cu -- the neural operator (a six-level convolutional U-Net) that
// predicts the steady morphogen field from the cell mask and source map and
// warm-starts the D2Q5 relaxation; forward, backward and Adam run in the
// kernels of nn.cu.  The paper has no network: this is the learned part the
// measured method adds on top of the steady solve.
//
// Definition (identical to the FP64 reference the tests compare with):
//   input   [cell mask, source mask, (D - 0.125)/0.075, log10(decay) + 3]
//   target  phi * decay / src_rate;  prediction phi = y * src_rate / decay
//   encoder level l = 0..5 (channels 32, 48, 64, 96, 128, 192):
//           conv3x3-ReLU-conv3x3-ReLU, 2x2 average pooling between levels
//   decoder level l = 4..0: conv3x3 on [skip_l, upsample2(deeper)] -ReLU-
//           conv3x3-ReLU; output conv3x3 to 1 channel; all with bias
//   loss    mean squared error; Adam (0.9, 0.999, 1e-8), bias-corrected
// Internally the input layer has 16 channels (12 zero) and the output layer
// 16 (15 zero); parameters are exchanged in the canonical flat layout
// (per layer weights (3,3,Ci,Co) then bias (Co)).
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbib_internal.cuh"
#include "nn.cuh"

using namespace lbib;
using bf16 = __nv_bfloat16;

namespace {

constexpr int kLevels = 6;
constexpr int kCh[kLevels] = {32, 48, 64, 96, 128, 192};
using nn::kConvSmem;
using nn::kTH;
using nn::kTW;
using nn::kWgSmem;

struct Layer {
    const char* name;
    int ci, co;      // canonical
    int cip, cop;    // internal (padded)
    int64_t off;     // offset in the internal FP32 parameter vector (weights, then bias)
    int64_t coff;    // offset in the canonical flat vector
    bf16* wf;        // (9, cop, cip)
    bf16* wd;        // (9, cip, cop)
    bf16* wft;       // wf tiled for the tcgen05 convolution
    bf16* wdt;       // wd tiled for the tcgen05 convolution (the data gradient)
};

std::vector<Layer> make_layers() {
    std::vector<Layer> L;
    auto add = [&](const char* nm, int ci, int co) {
        Layer l;
        l.name = nm;
        l.ci = ci;
        l.co = co;
        l.cip = ci < 16 ? 16 : ci;
        l.cop = co < 16 ? 16 : co;
        l.off = l.coff = 0;
        l.wf = l.wd = l.wft = l.wdt = nullptr;
        L.push_back(l);
    };
    static const char* enc_names[kLevels][2] = {{"enc0a", "enc0b"}, {"enc1a", "enc1b"},
                                                {"enc2a", "enc2b"}, {"enc3a", "enc3b"},
                                                {"enc4a", "enc4b"}, {"enc5a", "enc5b"}};
    static const char* dec_names[kLevels - 1][2] = {{"dec0a", "dec0b"}, {"dec1a", "dec1b"},
                                                    {"dec2a", "dec2b"}, {"dec3a", "dec3b"},
                                                    {"dec4a", "dec4b"}};
    int prev = 4;
    for (int l = 0; l < kLevels; ++l) {
        add(enc_names[l][0], prev, kCh[l]);
        add(enc_names[l][1], kCh[l], kCh[l]);
        prev = kCh[l];
    }
    for (int l = kLevels - 2; l >= 0; --l) {
        add(dec_names[l][0], kCh[l] + kCh[l + 1], kCh[l]);
        add(dec_names[l][1], kCh[l], kCh[l]);
    }
    add("out", kCh[0], 1);
    int64_t o = 0, co = 0;
    for (auto& l : L) {
        l.off = o;
        o += 9LL * l.cip * l.cop + l.cop;
        l.coff = co;
        co += 9LL * l.ci * l.co + l.co;
    }
    return L;
}

int64_t internal_params(const std::vector<Layer>& L) {
    const Layer& b = L.back();
    return b.off + 9LL * b.cip * b.cop + b.cop;
}
int64_t canonical_params(const std::vector<Layer>& L) {
    const Layer& b = L.back();
    return b.coff + 9LL * b.ci * b.co + b.co;
}

}  // namespace

struct lbib_nop {
    int B = 0, H = 0, W = 0;
    cudaStream_t stream = nullptr;
    char* ws = nullptr;
    uint64_t bytes = 0, used = 0;
    std::vector<Layer> L;
    int64_t P = 0;  // internal parameter count
    float *param = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    bf16 *x = nullptr, *dy = nullptr;
    bf16 *enc_in[kLevels], *enc_r1[kLevels], *enc_out[kLevels];
    bf16 *dec_r1[kLevels - 1], *dec_out[kLevels - 1], *gskip[kLevels - 1];
    bf16 *ga = nullptr, *gb = nullptr, *gc = nullptr;  // gradient scratch
    float* y = nullptr;      // (B, H, W, 16)
    float* tgt = nullptr;    // (B, H, W) scaled target
    float* fac = nullptr;    // per sample factor
    float* dn = nullptr;     // per sample normalised D, decay
    float* kn = nullptr;
    double* loss = nullptr;
    unsigned* tc_err = nullptr;  // raised by a tcgen05 convolution whose bounded wait ran out
    WeightSet* wsets = nullptr;  // per layer: master weights and their BF16 copies (device table)
    int64_t wsets_max = 0;       // the largest layer's element count over all its copies
    int64_t t = 0;           // Adam step
    std::string err;
    // pinned host staging: the per-sample inputs (3 B floats), then the loss
    // and the tensor-core status word of the last call, so that a call waits
    // on its stream once, at its end
    unsigned char* hpin = nullptr;
    bool pin_busy = false;  // copies out of hpin may be in flight (a call ended early)
    float* h_in() { return reinterpret_cast<float*>(hpin); }
    double* h_loss() { return reinterpret_cast<double*>(hpin + pin_off()); }
    unsigned* h_err() { return reinterpret_cast<unsigned*>(hpin + pin_off() + 8); }
    size_t pin_off() const { return ((size_t)3 * B * 4 + 15) / 16 * 16; }
    size_t pin_bytes() const { return pin_off() + 16; }
    ~lbib_nop() {
        if (hpin) cudaFreeHost(hpin);
    }

    template <typename T>
    T* take(uint64_t count) {
        uint64_t at = (used + 255) / 256 * 256;
        used = at + count * sizeof(T);
        return ws ? reinterpret_cast<T*>(ws + at) : nullptr;
    }
};

namespace {

static thread_local std::string g_nop_err;

int nop_fail(lbib_nop* n, int code, const std::string& msg) {
    if (n) n->err = msg;
    g_nop_err = msg;
    set_thread_error(code, msg);
    return code;
}

// lay the buffers out (with ws == nullptr: only count the bytes)
void nop_layout(lbib_nop* n) {
    n->used = 0;
    n->L = make_layers();
    n->P = internal_params(n->L);
    n->param = n->take<float>(n->P);
    n->grad = n->take<float>(n->P);
    n->m = n->take<float>(n->P);
    n->v = n->take<float>(n->P);
    for (auto& l : n->L) {
        l.wf = n->take<bf16>(9LL * l.cip * l.cop);
        l.wd = n->take<bf16>(9LL * l.cip * l.cop);
        l.wft = n->take<bf16>(tc_tiled_weight_elems(l.cip, l.cop));
        l.wdt = n->take<bf16>(tc_tiled_weight_elems(l.cop, l.cip));
    }
    n->tc_err = n->take<unsigned>(1);
    n->wsets = n->take<WeightSet>(n->L.size());
    const int64_t B = n->B;
    int64_t maxg = 0;
    for (int l = 0; l < kLevels; ++l) {
        const int64_t hw = (int64_t)(n->H >> l) * (n->W >> l);
        const int cin = l == 0 ? 16 : kCh[l - 1];
        n->enc_in[l] = n->take<bf16>(B * hw * cin);
        n->enc_r1[l] = n->take<bf16>(B * hw * kCh[l]);
        n->enc_out[l] = n->take<bf16>(B * hw * kCh[l]);
        if (l < kLevels - 1) {
            n->dec_r1[l] = n->take<bf16>(B * hw * kCh[l]);
            n->dec_out[l] = n->take<bf16>(B * hw * kCh[l]);
            n->gskip[l] = n->take<bf16>(B * hw * kCh[l]);
            maxg = std::max(maxg, B * hw * (kCh[l] + kCh[l + 1]));
        }
        maxg = std::max(maxg, B * hw * (int64_t)kCh[l]);
    }
    n->x = n->enc_in[0];
    n->ga = n->take<bf16>(maxg);
    n->gb = n->take<bf16>(maxg);
    n->gc = n->take<bf16>(maxg);
    n->dy = n->take<bf16>(B * n->H * n->W * 16);
    n->y = n->take<float>(B * n->H * n->W * 16);
    n->tgt = n->take<float>(B * n->H * n->W);
    n->fac = n->take<float>(B);
    n->dn = n->take<float>(B);
    n->kn = n->take<float>(B);
    n->loss = n->take<double>(1);
}

inline unsigned blocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// A 3x3 convolution of the network: on the tcgen05 tensor cores (tiled
// weights wt) for images of rows of 128 pixels or more, where the single
// halo per tile makes them the faster kernel (1.7 - 2.4x at 256 x 256, even
// at 128 x 128); narrower levels, where the three kx-shifted halo copies
// cost more than the warp-level kernel's register tiling, take the latter.
cudaError_t conv_fwd(lbib_nop* n, const Layer& l, const bf16* in1, const bf16* in2, int C1, int C2,
                     int lvl, void* out, int relu, int out_f32, const bf16* w, const bf16* wt,
                     const float* bias, int Co, int N, const bf16* gate = nullptr) {
    NvtxRange nvtx_range("nn.conv3x3");
    nn::ConvArgs a;
    a.in1 = in1;
    a.in2 = in2;
    a.w = w;
    a.bias = bias;
    a.out = out;
    a.N = N;
    a.H = n->H >> lvl;
    a.W = n->W >> lvl;
    a.C1 = C1;
    a.C2 = C2;
    a.Co = Co;
    a.relu = relu;
    a.out_f32 = out_f32;
    a.gate = gate;
    (void)l;
    if (wt && a.W >= 128 && tc_conv_supported(a.H, a.W, C1, C2, Co)) return tc_conv3x3(a, wt, n->tc_err, n->stream);
    const int tiles = ((a.H + kTH - 1) / kTH) * ((a.W + kTW - 1) / kTW);
    dim3 grid(tiles, (Co + 63) / 64, N);
    nn::conv3x3_fwd_kernel<<<grid, 256, kConvSmem, n->stream>>>(a);
    return cudaGetLastError();
}

cudaError_t conv_wgrad(lbib_nop* n, const Layer& l, const bf16* in1, const bf16* in2, int C1,
                       int C2, int lvl, const bf16* g, int N) {
    NvtxRange nvtx_range("nn.conv3x3_wgrad");
    nn::WgradArgs a;
    a.in1 = in1;
    a.in2 = in2;
    a.g = g;
    a.dw = n->grad + l.off;
    a.db = n->grad + l.off + 9LL * l.cip * l.cop;
    a.N = N;
    a.H = n->H >> lvl;
    a.W = n->W >> lvl;
    a.C1 = C1;
    a.C2 = C2;
    a.Co = l.cop;
    // the tcgen05 kernel wherever it measured faster (batch 16): every level
    // it supports (W >= 16) except the plain 16^2 layers
    const bool tc = tc_wgrad_supported(a.H, a.W, C1, C2, a.Co) && (a.W >= 32 || C2 > 0);
    if (tc) return tc_conv3x3_wgrad(a, n->tc_err, n->stream);
    const int tiles = ((a.H + kTH - 1) / kTH) * ((a.W + kTW - 1) / kTW) * N;
    a.tiles_per_cta = tiles > 4096 ? 32 : (tiles > 512 ? 8 : 1);
    dim3 grid((tiles + a.tiles_per_cta - 1) / a.tiles_per_cta, (C1 + C2 + 15) / 16, (l.cop + 63) / 64);
    nn::conv3x3_wgrad_kernel<<<grid, 256, kWgSmem, n->stream>>>(a);
    return cudaGetLastError();
}

// The BF16 copies of every layer's weights (forward, tap-flipped, and their
// tcgen05 tilings) from the FP32 master weights, in one launch.
cudaError_t refresh_weights(lbib_nop* n) {
    return refresh_weight_sets(n->wsets, (int)n->L.size(), n->wsets_max, n->stream);
}

cudaError_t set_inputs(lbib_nop* n, int N, const uint8_t* mask, const uint8_t* src,
                       const double* D, const double* decay, const double* src_rate,
                       bool target_scale) {
    // the pinned staging buffer: the previous call's copies out of it ended
    // with that call's wait on the stream, unless it ended early
    if (n->pin_busy) {
        const cudaError_t w = cudaStreamSynchronize(n->stream);
        if (w != cudaSuccess) return w;
    }
    n->pin_busy = true;
    float* h = n->h_in();
    for (int i = 0; i < N; ++i) {
        h[i] = (float)((D[i] - 0.125) / 0.075);
        h[N + i] = (float)(std::log10(decay[i]) + 3.0);
        // target: phi * decay / src; prediction: y * src / decay
        h[2 * N + i] = (float)(target_scale ? decay[i] / src_rate[i] : src_rate[i] / decay[i]);
    }
    cudaError_t e = cudaMemcpyAsync(n->dn, h, N * 4, cudaMemcpyHostToDevice, n->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(n->kn, h + N, N * 4, cudaMemcpyHostToDevice, n->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(n->fac, h + 2 * N, N * 4, cudaMemcpyHostToDevice, n->stream);
    if (e != cudaSuccess) return e;
    const int HW = n->H * n->W;
    nn::features_kernel<<<blocks((int64_t)N * HW), 256, 0, n->stream>>>(mask, src, n->dn, n->kn,
                                                                         n->x, N, HW);
    return cudaGetLastError();
}

cudaError_t forward(lbib_nop* n, int N) {
    cudaError_t e = cudaSuccess;
    const std::vector<Layer>& L = n->L;
    int li = 0;
    for (int l = 0; l < kLevels && e == cudaSuccess; ++l) {
        const int64_t hw = (int64_t)(n->H >> l) * (n->W >> l);
        if (l > 0) {
            nn::avgpool2_kernel<<<blocks(N * hw * kCh[l - 1] / 8), 256, 0, n->stream>>>(
                n->enc_out[l - 1], n->enc_in[l], N, n->H >> (l - 1), n->W >> (l - 1), kCh[l - 1]);
            e = cudaGetLastError();
        }
        const int cin = l == 0 ? 16 : kCh[l - 1];
        const Layer& a = L[li++];
        const Layer& b = L[li++];
        if (e == cudaSuccess)
            e = conv_fwd(n, a, n->enc_in[l], nullptr, cin, 0, l, n->enc_r1[l], 1, 0, a.wf, a.wft,
                         n->param + a.off + 9LL * a.cip * a.cop, a.cop, N);
        if (e == cudaSuccess)
            e = conv_fwd(n, b, n->enc_r1[l], nullptr, kCh[l], 0, l, n->enc_out[l], 1, 0, b.wf, b.wft,
                         n->param + b.off + 9LL * b.cip * b.cop, b.cop, N);
    }
    for (int l = kLevels - 2; l >= 0 && e == cudaSuccess; --l) {
        const Layer& a = L[li++];
        const Layer& b = L[li++];
        const bf16* deeper = (l == kLevels - 2) ? n->enc_out[l + 1] : n->dec_out[l + 1];
        e = conv_fwd(n, a, n->enc_out[l], deeper, kCh[l], kCh[l + 1], l, n->dec_r1[l], 1, 0, a.wf, a.wft,
                     n->param + a.off + 9LL * a.cip * a.cop, a.cop, N);
        if (e == cudaSuccess)
            e = conv_fwd(n, b, n->dec_r1[l], nullptr, kCh[l], 0, l, n->dec_out[l], 1, 0, b.wf, b.wft,
                         n->param + b.off + 9LL * b.cip * b.cop, b.cop, N);
    }
    if (e == cudaSuccess) {
        const Layer& o = L[li];
        e = conv_fwd(n, o, n->dec_out[0], nullptr, kCh[0], 0, 0, n->y, 0, 1, o.wf, o.wft,
                     n->param + o.off + 9LL * o.cip * o.cop, o.cop, N);
    }
    return e;
}

cudaError_t backward(lbib_nop* n, int N) {
    const std::vector<Layer>& L = n->L;
    cudaError_t e = cudaMemsetAsync(n->grad, 0, n->P * 4, n->stream);
    // layer indices: enc l a/b = 2l, 2l+1; dec l a/b = 12 + 2(4 - l), +1; out = 22
    auto enc = [&](int l, int ab) -> const Layer& { return L[2 * l + ab]; };
    auto dec = [&](int l, int ab) -> const Layer& { return L[12 + 2 * (kLevels - 2 - l) + ab]; };
    const Layer& o = L[22];
    const int64_t hw0 = (int64_t)n->H * n->W;
    // output layer
    if (e == cudaSuccess) e = conv_wgrad(n, o, n->dec_out[0], nullptr, kCh[0], 0, 0, n->dy, N);
    // every ReLU backward is fused into the kernel that produces the gradient
    // (the data-gradient convolutions, the concatenation split, the skip sum)
    if (e == cudaSuccess)
        e = conv_fwd(n, o, n->dy, nullptr, o.cop, 0, 0, n->ga, 0, 0, o.wd, o.wdt, nullptr, o.cip, N,
                     n->dec_out[0]);
    bf16* g = n->ga;
    bf16* s1 = n->gb;
    bf16* s2 = n->gc;
    for (int l = 0; l < kLevels - 1 && e == cudaSuccess; ++l) {
        const int64_t hw = (int64_t)(n->H >> l) * (n->W >> l);
        const Layer& a = dec(l, 0);
        const Layer& b = dec(l, 1);
        if (e == cudaSuccess) e = conv_wgrad(n, b, n->dec_r1[l], nullptr, kCh[l], 0, l, g, N);
        if (e == cudaSuccess)
            e = conv_fwd(n, b, g, nullptr, kCh[l], 0, l, s1, 0, 0, b.wd, b.wdt, nullptr, kCh[l], N,
                         n->dec_r1[l]);
        const bf16* deeper = (l == kLevels - 2) ? n->enc_out[l + 1] : n->dec_out[l + 1];
        if (e == cudaSuccess)
            e = conv_wgrad(n, a, n->enc_out[l], deeper, kCh[l], kCh[l + 1], l, s1, N);
        if (e == cudaSuccess)
            e = conv_fwd(n, a, s1, nullptr, kCh[l], 0, l, s2, 0, 0, a.wd, a.wdt,
                         nullptr, kCh[l] + kCh[l + 1], N);
        if (e == cudaSuccess) {
            const int64_t tot = (N * hw * kCh[l] + N * (hw / 4) * kCh[l + 1]) / 8;
            // g: the gradient of the deeper output, through its ReLU
            nn::concat_bwd_kernel<<<blocks(tot), 256, 0, n->stream>>>(
                s2, n->gskip[l], g, deeper, N, n->H >> l, n->W >> l, kCh[l], kCh[l + 1], 0);
            e = cudaGetLastError();
        }
        (void)hw0;
    }
    // g: gradient of the deepest encoder output (level 5)
    for (int l = kLevels - 1; l >= 0 && e == cudaSuccess; --l) {
        const int64_t hw = (int64_t)(n->H >> l) * (n->W >> l);
        const Layer& a = enc(l, 0);
        const Layer& b = enc(l, 1);
        if (l < kLevels - 1) {
            // the skip's gradient joins the deeper path's, through the ReLU
            // (at the deepest level the concatenation split applied it)
            nn::add_gate_kernel<<<blocks(N * hw * kCh[l] / 8), 256, 0, n->stream>>>(
                g, n->gskip[l], n->enc_out[l], N * hw * kCh[l]);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = conv_wgrad(n, b, n->enc_r1[l], nullptr, kCh[l], 0, l, g, N);
        if (e == cudaSuccess)
            e = conv_fwd(n, b, g, nullptr, kCh[l], 0, l, s1, 0, 0, b.wd, b.wdt, nullptr, kCh[l], N,
                         n->enc_r1[l]);
        const int cin = l == 0 ? 16 : kCh[l - 1];
        if (e == cudaSuccess) e = conv_wgrad(n, a, n->enc_in[l], nullptr, cin, 0, l, s1, N);
        if (l > 0 && e == cudaSuccess) {
            e = conv_fwd(n, a, s1, nullptr, kCh[l], 0, l, s2, 0, 0, a.wd, a.wdt, nullptr, cin, N);
            if (e == cudaSuccess) {
                const int64_t cnt = N * (int64_t)(n->H >> (l - 1)) * (n->W >> (l - 1)) * cin;
                nn::avgpool2_bwd_kernel<<<blocks(cnt / 8), 256, 0, n->stream>>>(
                    s2, g, N, n->H >> (l - 1), n->W >> (l - 1), cin);
                e = cudaGetLastError();
            }
        }
    }
    return e;
}

bool params_ok(lbib_nop* n) { return n && n->param; }

// After the stream has been synchronised: whether a tcgen05 convolution's
// bounded wait ran out since the last check (the word is then cleared).
// the end of a call: the status word back with the call's other results,
// one wait on the stream
int tc_status(lbib_nop* n, const char* where) {
    cudaError_t e = cudaMemcpyAsync(n->h_err(), n->tc_err, 4, cudaMemcpyDeviceToHost, n->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    if (e == cudaSuccess) n->pin_busy = false;
    const unsigned h = e == cudaSuccess ? *n->h_err() : 0u;
    if (e == cudaSuccess && h) {
        e = cudaMemsetAsync(n->tc_err, 0, 4, n->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    }
    if (e != cudaSuccess) return nop_fail(n, LBIB_E_CUDA, cudaGetErrorString(e));
    if (h)
        return nop_fail(n, LBIB_E_TIMEOUT,
                        std::string(where) + ": a tensor-core convolution's wait ran out");
    return LBIB_OK;
}

}  // namespace

extern "C" {

int lbib_nop_workspace_size(int32_t batch, int32_t H, int32_t W, uint64_t* bytes_out) {
    if (batch < 1 || H < 32 || W < 32 || H % 32 || W % 32 || !bytes_out)
        return nop_fail(nullptr, LBIB_E_PARAM,
                        "lbib_nop_workspace_size: batch >= 1, H and W multiples of 32");
    lbib_nop tmp;
    tmp.B = batch;
    tmp.H = H;
    tmp.W = W;
    nop_layout(&tmp);
    *bytes_out = tmp.used + 256;
    return LBIB_OK;
}

int lbib_nop_create(int32_t batch, int32_t H, int32_t W, void* d_workspace, uint64_t bytes,
                    void* cuda_stream, lbib_nop** out) {
    if (!out) return nop_fail(nullptr, LBIB_E_PARAM, "out is NULL");
    *out = nullptr;
    uint64_t need = 0;
    int rc = lbib_nop_workspace_size(batch, H, W, &need);
    if (rc) return rc;
    if (!d_workspace || bytes < need || reinterpret_cast<uintptr_t>(d_workspace) % 256)
        return nop_fail(nullptr, LBIB_E_WORKSPACE,
                        "lbib_nop_create: workspace NULL, misaligned or below " + std::to_string(need));
    lbib_nop* n = new (std::nothrow) lbib_nop();
    if (!n) return nop_fail(nullptr, LBIB_E_PARAM, "out of host memory");
    n->B = batch;
    n->H = H;
    n->W = W;
    n->ws = static_cast<char*>(d_workspace);
    n->bytes = bytes;
    n->stream = static_cast<cudaStream_t>(cuda_stream);
    nop_layout(n);
    cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&n->hpin), n->pin_bytes(),
                                  cudaHostAllocDefault);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(nn::conv3x3_fwd_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kConvSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(nn::conv3x3_wgrad_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kWgSmem);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->param, 0, n->P * 4 * 4, n->stream);  // param, grad, m, v
    if (e == cudaSuccess) e = cudaMemsetAsync(n->tc_err, 0, 4, n->stream);
    std::vector<WeightSet> sets;
    for (const Layer& l : n->L) {
        WeightSet w;
        w.w = n->param + l.off;
        w.wf = l.wf;
        w.wd = l.wd;
        w.wft = l.wft;
        w.wdt = l.wdt;
        w.Ci = l.cip;
        w.Co = l.cop;
        sets.push_back(w);
        n->wsets_max = std::max(n->wsets_max, weight_set_elems(l.cip, l.cop));
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(n->wsets, sets.data(), sets.size() * sizeof(WeightSet),
                            cudaMemcpyHostToDevice, n->stream);
    if (e == cudaSuccess) e = refresh_weights(n);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    if (e != cudaSuccess) {
        delete n;
        return nop_fail(nullptr, LBIB_E_CUDA, std::string("lbib_nop_create: ") + cudaGetErrorString(e));
    }
    *out = n;
    return LBIB_OK;
}

int lbib_nop_num_params(const lbib_nop* n, int64_t* count) {
    if (!n || !count) return LBIB_E_PARAM;
    *count = canonical_params(n->L);
    return LBIB_OK;
}

int lbib_nop_layers(const lbib_nop* n, int32_t* n_layers, int32_t* ci_co) {
    if (!n || !n_layers) return LBIB_E_PARAM;
    *n_layers = (int32_t)n->L.size();
    if (ci_co)
        for (size_t i = 0; i < n->L.size(); ++i) {
            ci_co[2 * i] = n->L[i].ci;
            ci_co[2 * i + 1] = n->L[i].co;
        }
    return LBIB_OK;
}

// canonical <-> internal parameter layouts (host side)
static void to_internal(const std::vector<Layer>& L, const float* canon, std::vector<float>& in) {
    in.assign((size_t)internal_params(L), 0.f);
    for (const auto& l : L) {
        for (int tap = 0; tap < 9; ++tap)
            for (int i = 0; i < l.ci; ++i)
                for (int o = 0; o < l.co; ++o)
                    in[l.off + ((int64_t)tap * l.cip + i) * l.cop + o] =
                        canon[l.coff + ((int64_t)tap * l.ci + i) * l.co + o];
        for (int o = 0; o < l.co; ++o)
            in[l.off + 9LL * l.cip * l.cop + o] = canon[l.coff + 9LL * l.ci * l.co + o];
    }
}
static void to_canonical(const std::vector<Layer>& L, const std::vector<float>& in, float* canon) {
    for (const auto& l : L) {
        for (int tap = 0; tap < 9; ++tap)
            for (int i = 0; i < l.ci; ++i)
                for (int o = 0; o < l.co; ++o)
                    canon[l.coff + ((int64_t)tap * l.ci + i) * l.co + o] =
                        in[l.off + ((int64_t)tap * l.cip + i) * l.cop + o];
        for (int o = 0; o < l.co; ++o)
            canon[l.coff + 9LL * l.ci * l.co + o] = in[l.off + 9LL * l.cip * l.cop + o];
    }
}

int lbib_nop_set_params(lbib_nop* n, const float* host, int64_t count) {
    if (!params_ok(n) || !host) return LBIB_E_PARAM;
    if (count != canonical_params(n->L)) return nop_fail(n, LBIB_E_PARAM, "parameter count mismatch");
    std::vector<float> in;
    to_internal(n->L, host, in);
    cudaError_t e = cudaMemcpyAsync(n->param, in.data(), in.size() * 4, cudaMemcpyHostToDevice, n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->m, 0, n->P * 4, n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->v, 0, n->P * 4, n->stream);
    if (e == cudaSuccess) e = refresh_weights(n);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    if (e != cudaSuccess) return nop_fail(n, LBIB_E_CUDA, cudaGetErrorString(e));
    n->t = 0;
    return LBIB_OK;
}

static int get_vec(lbib_nop* n, const float* dev, float* host, int64_t count) {
    if (!params_ok(n) || !host) return LBIB_E_PARAM;
    if (count != canonical_params(n->L)) return nop_fail(n, LBIB_E_PARAM, "parameter count mismatch");
    std::vector<float> in((size_t)n->P);
    cudaError_t e = cudaMemcpyAsync(in.data(), dev, n->P * 4, cudaMemcpyDeviceToHost, n->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    if (e != cudaSuccess) return nop_fail(n, LBIB_E_CUDA, cudaGetErrorString(e));
    to_canonical(n->L, in, host);
    return LBIB_OK;
}

int lbib_nop_get_params(lbib_nop* n, float* host, int64_t count) {
    return get_vec(n, n ? n->param : nullptr, host, count);
}
int lbib_nop_get_grads(lbib_nop* n, float* host, int64_t count) {
    return get_vec(n, n ? n->grad : nullptr, host, count);
}

int lbib_nop_forward(lbib_nop* n, int32_t N, const uint8_t* d_mask, const uint8_t* d_src,
                     const double* D, const double* decay, const double* src_rate, float* d_phi) {
    NvtxRange nvtx_range("lbib_nop_forward");
    if (!params_ok(n) || N < 1 || N > n->B || !d_mask || !d_src || !D || !decay || !src_rate ||
        !d_phi)
        return nop_fail(n, LBIB_E_PARAM, "lbib_nop_forward: invalid arguments");
    cudaError_t e = set_inputs(n, N, d_mask, d_src, D, decay, src_rate, false);
    if (e == cudaSuccess) e = forward(n, N);
    if (e == cudaSuccess) {
        const int HW = n->H * n->W;
        nn::scale_kernel<<<blocks((int64_t)N * HW), 256, 0, n->stream>>>(n->y, 16, d_phi, n->fac, N, HW);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return nop_fail(n, LBIB_E_CUDA, cudaGetErrorString(e));
    return tc_status(n, "lbib_nop_forward");  // waits on the stream
}

int lbib_nop_train_step(lbib_nop* n, int32_t N, const uint8_t* d_mask, const uint8_t* d_src,
                        const double* D, const double* decay, const double* src_rate,
                        const float* d_phi_target, double lr, int32_t update,
                        double* loss_out) {
    NvtxRange nvtx_range("lbib_nop_train_step");
    if (!params_ok(n) || N < 1 || N > n->B || !d_mask || !d_src || !D || !decay || !src_rate ||
        !d_phi_target)
        return nop_fail(n, LBIB_E_PARAM, "lbib_nop_train_step: invalid arguments");
    cudaError_t e = set_inputs(n, N, d_mask, d_src, D, decay, src_rate, true);
    const int HW = n->H * n->W;
    const int64_t np = (int64_t)N * HW;
    if (e == cudaSuccess) {
        nn::scale_kernel<<<blocks(np), 256, 0, n->stream>>>(d_phi_target, 1, n->tgt, n->fac, N, HW);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = forward(n, N);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->loss, 0, 8, n->stream);
    if (e == cudaSuccess) {
        nn::mse_kernel<<<blocks(np), 256, 0, n->stream>>>(n->y, 16, n->tgt, n->dy, 16, np, n->loss);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = backward(n, N);
    if (e == cudaSuccess && update) {
        n->t += 1;
        const float c1 = (float)(1.0 - std::pow(0.9, (double)n->t));
        const float c2 = (float)(1.0 - std::pow(0.999, (double)n->t));
        nn::adam_kernel<<<blocks(n->P), 256, 0, n->stream>>>(n->param, n->grad, n->m, n->v, n->P,
                                                             (float)lr, 0.9f, 0.999f, 1e-8f, c1, c2);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = refresh_weights(n);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(n->h_loss(), n->loss, 8, cudaMemcpyDeviceToHost, n->stream);
    if (e != cudaSuccess) return nop_fail(n, LBIB_E_CUDA, cudaGetErrorString(e));
    const int rc = tc_status(n, "lbib_nop_train_step");  // waits on the stream
    if (loss_out && rc != LBIB_E_CUDA) *loss_out = *n->h_loss();
    return rc;
}

void lbib_nop_destroy(lbib_nop* n) { delete n; }

const char* lbib_nop_last_error(const lbib_nop* n) { return n ? n->err.c_str() : g_nop_err.c_str(); }

// ---- single convolution layers (device pointers), for tests and users
int lbib_nn_conv3x3(int32_t N, int32_t H, int32_t W, int32_t C1, int32_t C2, int32_t Co,
                    const void* d_in1, const void* d_in2, const void* d_wf, const float* d_bias,
                    void* d_out, int32_t relu, int32_t out_f32, void* cuda_stream) {
    if (N < 1 || H < 1 || W < 1 || C1 % 16 || C2 % 16 || C1 < 16 || Co < 2 || Co % 2 || !d_in1 ||
        !d_wf || !d_out || (C2 > 0 && (!d_in2 || H % 2 || W % 2)))
        return set_thread_error(LBIB_E_PARAM, "lbib_nn_conv3x3: invalid arguments");
    nn::ConvArgs a;
    a.in1 = static_cast<const bf16*>(d_in1);
    a.in2 = static_cast<const bf16*>(d_in2);
    a.w = static_cast<const bf16*>(d_wf);
    a.bias = d_bias;
    a.out = d_out;
    a.N = N;
    a.H = H;
    a.W = W;
    a.C1 = C1;
    a.C2 = C2;
    a.Co = Co;
    a.relu = relu;
    a.out_f32 = out_f32;
    a.gate = nullptr;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaFuncSetAttribute(nn::conv3x3_fwd_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kConvSmem);
    if (e == cudaSuccess) {
        const int tiles = ((H + kTH - 1) / kTH) * ((W + kTW - 1) / kTW);
        nn::conv3x3_fwd_kernel<<<dim3(tiles, (Co + 63) / 64, N), 256, kConvSmem, st>>>(a);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return set_thread_error(LBIB_E_CUDA, cudaGetErrorString(e));
    return LBIB_OK;
}

int lbib_nn_conv3x3_tc_supported(int32_t H, int32_t W, int32_t C1, int32_t C2, int32_t Co) {
    return tc_conv_supported(H, W, C1, C2, Co) ? 1 : 0;
}

int lbib_nn_tile_weights_tc(int32_t Ci, int32_t Co, const void* d_wf, void* d_wt,
                            uint64_t* elems_out, void* cuda_stream) {
    if (Ci < 16 || Ci % 16 || Co < 1)
        return set_thread_error(LBIB_E_PARAM, "lbib_nn_tile_weights_tc: invalid arguments");
    if (elems_out) *elems_out = (uint64_t)tc_tiled_weight_elems(Ci, Co);
    if (!d_wt) return LBIB_OK;
    if (!d_wf) return set_thread_error(LBIB_E_PARAM, "lbib_nn_tile_weights_tc: d_wf is NULL");
    cudaError_t e = tc_tile_weights(d_wf, Co, Ci, d_wt, static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return set_thread_error(LBIB_E_CUDA, cudaGetErrorString(e));
    return LBIB_OK;
}

int lbib_nn_conv3x3_tc(int32_t N, int32_t H, int32_t W, int32_t C1, int32_t C2, int32_t Co,
                       const void* d_in1, const void* d_in2, const void* d_wt, const float* d_bias,
                       void* d_out, int32_t relu, int32_t out_f32, uint32_t* d_err,
                       void* cuda_stream) {
    if (N < 1 || !d_in1 || !d_wt || !d_out || !d_err || (C2 > 0 && !d_in2) ||
        !tc_conv_supported(H, W, C1, C2, Co))
        return set_thread_error(LBIB_E_PARAM, "lbib_nn_conv3x3_tc: unsupported shape or arguments");
    if (reinterpret_cast<uintptr_t>(d_in1) % 16 || reinterpret_cast<uintptr_t>(d_wt) % 16 ||
        reinterpret_cast<uintptr_t>(d_out) % 16 || (d_in2 && reinterpret_cast<uintptr_t>(d_in2) % 16))
        return set_thread_error(LBIB_E_PARAM, "lbib_nn_conv3x3_tc: buffers need 16-byte alignment");
    nn::ConvArgs a;
    a.in1 = static_cast<const bf16*>(d_in1);
    a.in2 = static_cast<const bf16*>(d_in2);
    a.w = nullptr;
    a.bias = d_bias;
    a.out = d_out;
    a.N = N;
    a.H = H;
    a.W = W;
    a.C1 = C1;
    a.C2 = C2;
    a.Co = Co;
    a.relu = relu;
    a.out_f32 = out_f32;
    a.gate = nullptr;
    cudaError_t e = tc_conv3x3(a, d_wt, d_err, static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return set_thread_error(LBIB_E_CUDA, cudaGetErrorString(e));
    return LBIB_OK;
}

int lbib_nn_conv3x3_wgrad_tc_supported(int32_t H, int32_t W, int32_t C1, int32_t C2, int32_t Co) {
    return tc_wgrad_supported(H, W, C1, C2, Co) ? 1 : 0;
}

int lbib_nn_conv3x3_wgrad_tc(int32_t N, int32_t H, int32_t W, int32_t C1, int32_t C2, int32_t Co,
                             const void* d_in1, const void* d_in2, const void* d_g, float* d_dw,
                             float* d_db, uint32_t* d_err, void* cuda_stream) {
    if (N < 1 || !d_in1 || !d_g || !d_dw || !d_err || (C2 > 0 && !d_in2) ||
        !tc_wgrad_supported(H, W, C1, C2, Co))
        return set_thread_error(LBIB_E_PARAM,
                                "lbib_nn_conv3x3_wgrad_tc: unsupported shape or arguments");
    if (reinterpret_cast<uintptr_t>(d_in1) % 16 || reinterpret_cast<uintptr_t>(d_g) % 16 ||
        reinterpret_cast<uintptr_t>(d_dw) % 16 || (d_in2 && reinterpret_cast<uintptr_t>(d_in2) % 16))
        return set_thread_error(LBIB_E_PARAM, "lbib_nn_conv3x3_wgrad_tc: buffers need 16-byte alignment");
    nn::WgradArgs a;
    std::memset(&a, 0, sizeof(a));
    a.in1 = static_cast<const bf16*>(d_in1);
    a.in2 = static_cast<const bf16*>(d_in2);
    a.g = static_cast<const bf16*>(d_g);
    a.dw = d_dw;
    a.db = d_db;
    a.N = N;
    a.H = H;
    a.W = W;
    a.C1 = C1;
    a.C2 = C2;
    a.Co = Co;
    cudaError_t e = tc_conv3x3_wgrad(a, d_err, static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return set_thread_error(LBIB_E_CUDA, cudaGetErrorString(e));
    return LBIB_OK;
}

int lbib_nn_conv3x3_wgrad(int32_t N, int32_t H, int32_t W, int32_t C1, int32_t C2, int32_t Co,
                          const void* d_in1, const void* d_in2, const void* d_g, float* d_dw,
                          float* d_db, void* cuda_stream) {
    if (N < 1 || H < 1 || W < 1 || C1 % 16 || C2 % 16 || C1 < 16 || Co % 8 || Co < 8 || !d_in1 ||
        !d_g || !d_dw || (C2 > 0 && (!d_in2 || H % 2 || W % 2)))
        return set_thread_error(LBIB_E_PARAM, "lbib_nn_conv3x3_wgrad: invalid arguments");
    nn::WgradArgs a;
    a.in1 = static_cast<const bf16*>(d_in1);
    a.in2 = static_cast<const bf16*>(d_in2);
    a.g = static_cast<const bf16*>(d_g);
    a.dw = d_dw;
    a.db = d_db;
    a.N = N;
    a.H = H;
    a.W = W;
    a.C1 = C1;
    a.C2 = C2;
    a.Co = Co;
    const int tiles = ((H + kTH - 1) / kTH) * ((W + kTW - 1) / kTW) * N;
    a.tiles_per_cta = 4;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaFuncSetAttribute(nn::conv3x3_wgrad_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kWgSmem);
    if (e == cudaSuccess) {
        dim3 grid((tiles + 3) / 4, (C1 + C2 + 15) / 16, (Co + 63) / 64);
        nn::conv3x3_wgrad_kernel<<<grid, 256, kWgSmem, st>>>(a);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return set_thread_error(LBIB_E_CUDA, cudaGetErrorString(e));
    return LBIB_OK;
}

int lbib_nn_weight_copies(int32_t Ci, int32_t Co, int32_t Cip, int32_t Cop, const float* d_w,
                          void* d_wf, void* d_wd, void* cuda_stream) {
    if (Ci < 1 || Co < 1 || Cip < Ci || Cop < Co || !d_w || !d_wf || !d_wd)
        return set_thread_error(LBIB_E_PARAM, "lbib_nn_weight_copies: invalid arguments");
    const int64_t cnt = 9LL * Cip * Cop;
    nn::weight_copies_kernel<<<blocks(cnt), 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
        d_w, Ci, Co, Cip, Cop, static_cast<bf16*>(d_wf), static_cast<bf16*>(d_wd));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_thread_error(LBIB_E_CUDA, cudaGetErrorString(e));
    return LBIB_OK;
}

}  // extern "C"
