// Agent network of a worker: parameter layout, weight preparation, the forward pass over
// a [T, E] segment (encoder -> visual FC -> goal/action embeddings -> L-layer LSTM ->
// actor/critic), and the hand-written backward (heads -> LSTM back-propagation through
// time -> embeddings -> visual FC -> encoder, with per-chunk recomputation when the
// encoder runs in several chunks). App. "Agent Design"; Sec. 4 "Agent".
#include <math.h>

#include <algorithm>

#include "net.cuh"
#include "nn_kernels.cuh"
#include "rl.cuh"

namespace ddppo {

template <class T>
static int nalloc(Net& n, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return DDPPO_OK;
  void* q = nullptr;
  DDPPO_CHECK_CUDA(cudaMalloc(&q, count * sizeof(T)));
  n.allocs.push_back(q);
  *p = (T*)q;
  return DDPPO_OK;
}
static int nalloc_op(Net& n, void** p, size_t count) {
  *p = nullptr;
  if (count == 0) return DDPPO_OK;
  const size_t es = n.bf ? 2 : 4;
  DDPPO_CHECK_CUDA(cudaMalloc(p, count * es));
  n.allocs.push_back(*p);
  return DDPPO_OK;
}
static inline size_t esz(const Net& n) { return n.bf ? 2 : 4; }
static inline void* opoff(const Net& n, const void* p, size_t elems) {
  return (void*)((const char*)p + elems * esz(n));
}

static int conv_out(int v, int k, int s, int p) { return (v + 2 * p - k) / s + 1; }

// ---------------------------------------------------------------- layout
struct Layout {
  int64_t off = 0;
  int64_t add(int64_t n) { int64_t o = off; off += n; return o; }
};

static void set_conv(ConvL& c, int cin, int cout, int k, int s, int p, bool bias, int H, int W,
                     Layout& lay) {
  c.cin = cin; c.cout = cout; c.k = k; c.s = s; c.p = p; c.bias = bias;
  c.H = H; c.W = W; c.Ho = conv_out(H, k, s, p); c.Wo = conv_out(W, k, s, p);
  c.Kp = (k * k * cin + 7) / 8 * 8;
  c.w_off = lay.add((int64_t)cout * cin * k * k);
  if (bias) c.b_off = lay.add(cout);
}
static void set_gn(GNL& g, int C, Layout& lay) {
  g.C = C;
  g.g_off = lay.add(C);
  g.b_off = lay.add(C);
}

static ConvGeom geom(const ConvL& c, int N) {
  ConvGeom g;
  g.N = N; g.H = c.H; g.W = c.W; g.C = c.cin; g.Ho = c.Ho; g.Wo = c.Wo; g.Cout = c.cout;
  g.k = c.k; g.s = c.s; g.p = c.p; g.K = c.k * c.k * c.cin; g.Kp = c.Kp;
  return g;
}

// ---------------------------------------------------------------- creation
static int build_layout(Net& n, Layout& lay) {
  const ddppo_config& c = n.x->cfg;
  n.inh = c.depth_h >> c.pool2x2;
  n.inw = c.depth_w >> c.pool2x2;
  if (n.kind == 0) {
    set_conv(n.nat[0], 1, 32, 8, 4, 0, true, n.inh, n.inw, lay);
    set_conv(n.nat[1], 32, 64, 4, 2, 0, true, n.nat[0].Ho, n.nat[0].Wo, lay);
    set_conv(n.nat[2], 64, 32, 3, 1, 0, true, n.nat[1].Ho, n.nat[1].Wo, lay);
    if (n.nat[2].Ho < 1 || n.nat[2].Wo < 1) {
      set_error("depth too small for the 3-layer encoder");
      return DDPPO_E_CONFIG;
    }
    for (auto& cv : n.nat) n.convs.push_back(&cv);
    n.featC = 32;
    n.featHW = n.nat[2].Ho * n.nat[2].Wo;
  } else if (n.kind == 2) {
    // blind agent (GPS+Compass only, Sec. 5): no visual encoder, no visual FC
    n.featC = 0;
    n.featHW = 0;
  } else if (n.kind >= 3) {
    // SE-ResNeXt50 (kind 3) / 101 (kind 4) with every layer's channels halved: stem and
    // max pool as the ResNet's; bottlenecks [3, 4, 6, 3] / [3, 4, 23, 3] of inner width
    // 2b 2^i (grouped 3x3 with 32 groups, the stride here) and output 4b 2^i; squeeze-
    // excite with reduction 16; then the 3x3 compression to 128 channels
    const int b = c.base_ch;
    set_conv(n.stem, 1, b, 7, 2, 3, false, n.inh, n.inw, lay);
    set_gn(n.stem_n, b, lay);
    n.convs.push_back(&n.stem);
    int H = (n.stem.Ho - 1) / 2 + 1, W = (n.stem.Wo - 1) / 2 + 1;
    int cin = b;
    const int counts[2][4] = {{3, 4, 6, 3}, {3, 4, 23, 3}};
    const int* cnt = counts[n.kind == 3 ? 0 : 1];
    n.sx.resize(cnt[0] + cnt[1] + cnt[2] + cnt[3]);
    for (int i = 0, bi = 0; i < 4; ++i)
      for (int r = 0; r < cnt[i]; ++r, ++bi) {
        SxL& X = n.sx[bi];
        const int mid = (2 * b) << i, cout = (4 * b) << i, st = (i > 0 && r == 0) ? 2 : 1;
        set_conv(X.c1, cin, mid, 1, 1, 0, false, H, W, lay);
        set_gn(X.n1, mid, lay);
        GConvL& g = X.c2;
        g.C = mid; g.cpg = mid / 32; g.s = st; g.H = H; g.W = W;
        g.Ho = conv_out(H, 3, st, 1); g.Wo = conv_out(W, 3, st, 1);
        g.w_off = lay.add((int64_t)mid * g.cpg * 9);
        set_gn(X.n2, mid, lay);
        set_conv(X.c3, mid, cout, 1, 1, 0, false, g.Ho, g.Wo, lay);
        set_gn(X.n3, cout, lay);
        X.C = cout; X.Cr = cout / 16; X.HW = g.Ho * g.Wo;
        X.se1_w = lay.add((int64_t)X.Cr * cout);
        X.se1_b = lay.add(X.Cr);
        X.se2_w = lay.add((int64_t)cout * X.Cr);
        X.se2_b = lay.add(cout);
        X.down = st != 1 || cin != cout;
        if (X.down) {
          set_conv(X.d, cin, cout, 1, st, 0, false, H, W, lay);
          set_gn(X.nd, cout, lay);
          n.convs.push_back(&X.d);
        }
        n.convs.push_back(&X.c1);
        n.convs.push_back(&X.c3);
        H = g.Ho; W = g.Wo; cin = cout;
      }
    if (H < 1 || W < 1) { set_error("depth too small for the SE-ResNeXt encoder"); return DDPPO_E_CONFIG; }
    set_conv(n.cmp, cin, 128, 3, 1, 1, false, H, W, lay);
    set_gn(n.cmp_n, 128, lay);
    n.convs.push_back(&n.cmp);
    n.featC = 128;
    n.featHW = n.cmp.Ho * n.cmp.Wo;
  } else {
    const int b = c.base_ch;
    set_conv(n.stem, 1, b, 7, 2, 3, false, n.inh, n.inw, lay);
    set_gn(n.stem_n, b, lay);
    n.convs.push_back(&n.stem);
    int H = (n.stem.Ho - 1) / 2 + 1, W = (n.stem.Wo - 1) / 2 + 1;  // max pool 3x3/2 pad 1
    int cin = b;
    const int widths[4] = {b, 2 * b, 4 * b, 8 * b};
    for (int li = 0, bi = 0; li < 4; ++li)
      for (int r = 0; r < 2; ++r, ++bi) {
        BlockL& B = n.blocks[bi];
        const int w = widths[li], s = (li > 0 && r == 0) ? 2 : 1;
        set_conv(B.c1, cin, w, 3, s, 1, false, H, W, lay);
        set_gn(B.n1, w, lay);
        set_conv(B.c2, w, w, 3, 1, 1, false, B.c1.Ho, B.c1.Wo, lay);
        set_gn(B.n2, w, lay);
        B.down = (s != 1 || cin != w);
        if (B.down) {
          set_conv(B.d, cin, w, 1, s, 0, false, H, W, lay);
          set_gn(B.nd, w, lay);
          n.convs.push_back(&B.d);
        }
        n.convs.push_back(&B.c1);
        n.convs.push_back(&B.c2);
        H = B.c1.Ho; W = B.c1.Wo; cin = w;
      }
    if (H < 1 || W < 1) { set_error("depth too small for the ResNet encoder"); return DDPPO_E_CONFIG; }
    set_conv(n.cmp, 8 * b, 128, 3, 1, 1, false, H, W, lay);
    set_gn(n.cmp_n, 128, lay);
    n.convs.push_back(&n.cmp);
    n.featC = 128;
    n.featHW = n.cmp.Ho * n.cmp.Wo;
  }
  n.F = n.featC * n.featHW;
  const int Hd = n.H;
  if (n.F > 0) {
    n.vis_w = lay.add((int64_t)Hd * n.F);
    n.vis_b = lay.add(Hd);
  }
  n.goal_w = lay.add(32 * 3);
  n.goal_b = lay.add(32);
  n.emb = lay.add(5 * 32);
  // LSTM input [visual FC (H, when there is an encoder) | goal FC (32) | embedding (32)]
  n.emb_col0 = n.F > 0 ? Hd : 0;
  n.In0 = n.emb_col0 + 64;
  // widest LSTM input (its gradient buffers): layer 0's, or H above it (the blind agent's
  // first layer is narrower than the others)
  n.InMax = std::max(n.In0, Hd);
  for (int l = 0; l < n.L; ++l) {
    LstmL& s = n.lstm[l];
    s.In = l == 0 ? n.In0 : Hd;
    s.wih = lay.add((int64_t)4 * Hd * s.In);
    s.whh = lay.add((int64_t)4 * Hd * Hd);
    s.bih = lay.add(4 * Hd);
    s.bhh = lay.add(4 * Hd);
  }
  n.actor_w = lay.add(4 * Hd);
  n.actor_b = lay.add(4);
  n.critic_w = lay.add(Hd);
  n.critic_b = lay.add(1);
  return DDPPO_OK;
}

// FP8 inference buffers: E4M3 copies of the act-time convolution inputs (E images), E4M3
// weights of every convolution whose input channels are a multiple of 64, and the scale /
// absolute-maximum slots (activations first, then weights)
static int alloc_f8(Net& n, int pool_hw) {
  const size_t E = n.E;
  int slot = 0;
  n.pool_slot = slot++;
  DDPPO_TRY(nalloc(n, &n.pool_f8, E * pool_hw * n.stem.cout));
  for (auto& B : n.blocks) {
    B.n1.f8_slot = slot++;
    B.y_slot = slot++;
    DDPPO_TRY(nalloc(n, &B.n1.out_f8, E * B.c1.Ho * B.c1.Wo * B.c1.cout));
    DDPPO_TRY(nalloc(n, &B.y_f8, E * B.c2.Ho * B.c2.Wo * B.c2.cout));
  }
  n.f8_act_slots = slot;
  std::vector<ConvL*> wq;
  for (ConvL* c : n.convs)
    if (c->cin % 64 == 0 && c->Kp == c->k * c->k * c->cin) wq.push_back(c);
  n.f8_slots = slot + (int)wq.size();
  DDPPO_TRY(nalloc(n, &n.f8_scale, (size_t)n.f8_slots));
  DDPPO_TRY(nalloc(n, &n.f8_amax, (size_t)n.f8_slots));
  DDPPO_TRY(nalloc(n, &n.f8_keep, 2 * (size_t)n.f8_act_slots));
  for (ConvL* c : wq) {
    DDPPO_TRY(nalloc(n, &c->wg8, (size_t)c->cout * c->Kp));
    c->w8_scale = n.f8_scale + slot;
    c->w8_amax = n.f8_amax + slot;
    ++slot;
  }
  // first act pass: activations carried at scale 1/8 (|x| up to 56); later passes use the
  // previous pass's maxima
  std::vector<float> init(n.f8_slots, 1.f);
  for (int i = 0; i < n.f8_act_slots; ++i) init[i] = 0.125f;
  DDPPO_CHECK_CUDA(cudaMemcpy(n.f8_scale, init.data(), init.size() * 4, cudaMemcpyHostToDevice));
  DDPPO_CHECK_CUDA(cudaMemset(n.f8_amax, 0, (size_t)n.f8_slots * 4));
  return DDPPO_OK;
}

static int alloc_encoder(Net& n) {
  const size_t NC = n.NC;
  auto conv_bufs = [&](ConvL& c) -> int {
    DDPPO_TRY(nalloc_op(n, &c.wg, (size_t)c.cout * c.Kp));
    DDPPO_TRY(nalloc_op(n, &c.wgT, (size_t)c.cout * c.Kp));
    DDPPO_TRY(nalloc(n, &c.dwg, (size_t)c.cout * c.Kp));
    DDPPO_TRY(nalloc(n, &c.z, NC * c.Ho * c.Wo * c.cout));
    // a stride-1 'same' convolution's input gradient is a convolution of its output
    // gradient with the flipped, channel-swapped kernel: no col2im round trip
    c.dgrad_as_conv = c.s == 1 && c.k % 2 == 1 && c.p == c.k / 2 && c.cout % 8 == 0;
    if (c.dgrad_as_conv) {
      DDPPO_TRY(nalloc_op(n, &c.wgR, (size_t)c.cin * c.k * c.k * c.cout));
      n.max_col = std::max(n.max_col, (size_t)c.H * c.W * c.k * c.k * c.cout);
    }
    n.max_col = std::max(n.max_col, (size_t)c.Ho * c.Wo * c.Kp);
    n.max_dz = std::max(n.max_dz, (size_t)c.Ho * c.Wo * c.cout);
    n.max_act = std::max(n.max_act, c.Ho * c.Wo * c.cout);
    n.max_act = std::max(n.max_act, c.H * c.W * c.cin);
    return DDPPO_OK;
  };
  auto gn_bufs = [&](GNL& g, int HW, bool out) -> int {
    DDPPO_TRY(nalloc(n, &g.mean, NC * g.C / 2));
    DDPPO_TRY(nalloc(n, &g.rstd, NC * g.C / 2));
    if (out) DDPPO_TRY(nalloc(n, &g.out, NC * HW * g.C));
    n.max_gnC = std::max(n.max_gnC, g.C);
    return DDPPO_OK;
  };
  if (n.kind == 0) {
    for (auto& c : n.nat) DDPPO_TRY(conv_bufs(c));
  } else if (n.kind == 1 || n.kind >= 3) {
    DDPPO_TRY(conv_bufs(n.stem));
    // the stem's full-resolution activation is only stored when its pool is not fused
    DDPPO_TRY(gn_bufs(n.stem_n, n.stem.Ho * n.stem.Wo, n.stem.cout % 4 != 0));
    const int ph = (n.stem.Ho - 1) / 2 + 1, pw = (n.stem.Wo - 1) / 2 + 1;
    DDPPO_TRY(nalloc(n, &n.pool, NC * ph * pw * n.stem.cout));
    if (n.bf) DDPPO_TRY(nalloc(n, &n.pool_bf, NC * ph * pw * n.stem.cout));
    DDPPO_TRY(nalloc(n, &n.pool_arg, NC * ph * pw * n.stem.cout));
    int maxC = 0, maxCr = 0;
    for (SxL& X : n.sx) {
      const int HWi = X.c1.H * X.c1.W;
      DDPPO_TRY(conv_bufs(X.c1));
      DDPPO_TRY(conv_bufs(X.c3));
      DDPPO_TRY(gn_bufs(X.n1, HWi, true));
      DDPPO_TRY(gn_bufs(X.n2, X.HW, true));
      DDPPO_TRY(gn_bufs(X.n3, X.HW, false));
      if (X.down) {
        DDPPO_TRY(conv_bufs(X.d));
        DDPPO_TRY(gn_bufs(X.nd, X.HW, false));
        DDPPO_TRY(nalloc(n, &X.sc, NC * X.HW * X.C));
      }
      const GConvL& g = X.c2;
      DDPPO_TRY(nalloc_op(n, &X.c2.wg, (size_t)g.C * g.cpg * 9));
      DDPPO_TRY(nalloc(n, &X.c2.z, NC * X.HW * g.C));
      if (n.bf) {
        DDPPO_TRY(nalloc(n, &X.n1.out_bf, NC * HWi * g.C));
        DDPPO_TRY(nalloc(n, &X.n2.out_bf, NC * X.HW * g.C));
        DDPPO_TRY(nalloc(n, &X.y_bf, NC * X.HW * X.C));
      }
      DDPPO_TRY(nalloc(n, &X.u, NC * X.HW * X.C));
      DDPPO_TRY(nalloc(n, &X.y, NC * X.HW * X.C));
      DDPPO_TRY(nalloc(n, &X.m, NC * X.C));
      DDPPO_TRY(nalloc(n, &X.a, NC * X.Cr));
      DDPPO_TRY(nalloc(n, &X.gate, NC * X.C));
      GConv gc{(int)NC, g.H, g.W, g.C, g.cpg, g.s, g.Ho, g.Wo};
      n.gw_part_elems = std::max(n.gw_part_elems,
                                 (size_t)gconv_wgrad_chunks(gc, n.gws.num_sms) * g.C * g.cpg * 9);
      maxC = std::max(maxC, X.C);
      maxCr = std::max(maxCr, X.Cr);
    }
    if (!n.sx.empty()) {
      DDPPO_TRY(nalloc(n, &n.gw_part, n.gw_part_elems));
      DDPPO_TRY(nalloc(n, &n.se_dg, NC * maxC));
      DDPPO_TRY(nalloc(n, &n.se_dq, NC * maxC));
      DDPPO_TRY(nalloc(n, &n.se_dm, NC * maxC));
      DDPPO_TRY(nalloc(n, &n.se_dh, NC * maxCr));
    }
    for (auto& B : n.blocks) {
      if (n.kind != 1) break;
      DDPPO_TRY(conv_bufs(B.c1));
      DDPPO_TRY(conv_bufs(B.c2));
      DDPPO_TRY(gn_bufs(B.n1, B.c1.Ho * B.c1.Wo, true));
      DDPPO_TRY(gn_bufs(B.n2, B.c2.Ho * B.c2.Wo, false));
      if (B.down) {
        DDPPO_TRY(conv_bufs(B.d));
        DDPPO_TRY(gn_bufs(B.nd, B.d.Ho * B.d.Wo, false));
      }
      DDPPO_TRY(nalloc(n, &B.y, NC * B.c2.Ho * B.c2.Wo * B.c2.cout));
      if (n.bf) {
        DDPPO_TRY(nalloc(n, &B.y_bf, NC * B.c2.Ho * B.c2.Wo * B.c2.cout));
        DDPPO_TRY(nalloc(n, &B.n1.out_bf, NC * B.c1.Ho * B.c1.Wo * B.c1.cout));
      }
    }
    DDPPO_TRY(conv_bufs(n.cmp));
    DDPPO_TRY(gn_bufs(n.cmp_n, n.featHW, true));
    if (n.f8) DDPPO_TRY(alloc_f8(n, ph * pw));
  }
  DDPPO_TRY(nalloc_op(n, &n.col, NC * n.max_col));
  DDPPO_TRY(nalloc(n, &n.dcol, NC * n.max_col));
  DDPPO_TRY(nalloc_op(n, &n.dzop, NC * n.max_dz));
  DDPPO_TRY(nalloc(n, &n.g0, NC * n.max_act));
  DDPPO_TRY(nalloc(n, &n.g1, NC * n.max_act));
  DDPPO_TRY(nalloc(n, &n.g2, NC * n.max_act));
  const int C = std::max(n.max_gnC, 64);
  DDPPO_TRY(nalloc(n, &n.gnp_g, NC * C));
  DDPPO_TRY(nalloc(n, &n.gnp_b, NC * C));
  if (n.kind == 1 || n.kind >= 3) {
    n.gnw.max_images = (int)NC;
    n.gnw.part_elems = gn_part_elems((int)NC, C);
    DDPPO_TRY(nalloc(n, &n.gnw.part, n.gnw.part_elems));
    DDPPO_TRY(nalloc(n, &n.gnw.cnt, NC));
    DDPPO_CHECK_CUDA(cudaMemset(n.gnw.cnt, 0, NC * sizeof(int)));
    DDPPO_TRY(nalloc(n, &n.gnw.cnt2, NC));
    DDPPO_CHECK_CUDA(cudaMemset(n.gnw.cnt2, 0, NC * sizeof(int)));
    DDPPO_TRY(nalloc(n, &n.gn_m1, NC * C / 2));
    DDPPO_TRY(nalloc(n, &n.gn_m2, NC * C / 2));
  }
  return DDPPO_OK;
}

static int init_params(Net& n, cudaStream_t s) {
  const uint64_t seed = n.x->cfg.seed;
  uint64_t stream = 0;
  auto unif = [&](int64_t off, int64_t cnt, float b) {
    return launch_init_uniform(n.params + off, (size_t)cnt, -b, b, seed, stream++, s);
  };
  auto conv_init = [&](ConvL& c) -> int {
    const int fan = c.cin * c.k * c.k;
    DDPPO_TRY(unif(c.w_off, (int64_t)c.cout * fan, sqrtf(6.0f / fan)));
    if (c.bias) DDPPO_TRY(launch_fill(n.params + c.b_off, c.cout, 0.f, s));
    return DDPPO_OK;
  };
  auto gn_init = [&](GNL& g) -> int {
    DDPPO_TRY(launch_fill(n.params + g.g_off, g.C, 1.f, s));
    DDPPO_TRY(launch_fill(n.params + g.b_off, g.C, 0.f, s));
    return DDPPO_OK;
  };
  if (n.kind == 0) {
    for (auto& c : n.nat) DDPPO_TRY(conv_init(c));
  } else if (n.kind == 1) {
    DDPPO_TRY(conv_init(n.stem));
    DDPPO_TRY(gn_init(n.stem_n));
    for (auto& B : n.blocks) {
      DDPPO_TRY(conv_init(B.c1)); DDPPO_TRY(gn_init(B.n1));
      DDPPO_TRY(conv_init(B.c2)); DDPPO_TRY(gn_init(B.n2));
      if (B.down) { DDPPO_TRY(conv_init(B.d)); DDPPO_TRY(gn_init(B.nd)); }
    }
    DDPPO_TRY(conv_init(n.cmp));
    DDPPO_TRY(gn_init(n.cmp_n));
  } else if (n.kind >= 3) {
    DDPPO_TRY(conv_init(n.stem));
    DDPPO_TRY(gn_init(n.stem_n));
    for (SxL& X : n.sx) {
      DDPPO_TRY(conv_init(X.c1)); DDPPO_TRY(gn_init(X.n1));
      const int fan = X.c2.cpg * 9;
      DDPPO_TRY(unif(X.c2.w_off, (int64_t)X.c2.C * fan, sqrtf(6.0f / fan)));
      DDPPO_TRY(gn_init(X.n2));
      DDPPO_TRY(conv_init(X.c3)); DDPPO_TRY(gn_init(X.n3));
      DDPPO_TRY(unif(X.se1_w, (int64_t)X.Cr * X.C, sqrtf(6.0f / X.C)));
      DDPPO_TRY(launch_fill(n.params + X.se1_b, X.Cr, 0.f, s));
      DDPPO_TRY(unif(X.se2_w, (int64_t)X.C * X.Cr, sqrtf(6.0f / X.Cr)));
      DDPPO_TRY(launch_fill(n.params + X.se2_b, X.C, 0.f, s));
      if (X.down) { DDPPO_TRY(conv_init(X.d)); DDPPO_TRY(gn_init(X.nd)); }
    }
    DDPPO_TRY(conv_init(n.cmp));
    DDPPO_TRY(gn_init(n.cmp_n));
  }
  const int Hd = n.H;
  if (n.F > 0) {
    DDPPO_TRY(unif(n.vis_w, (int64_t)Hd * n.F, sqrtf(6.0f / n.F)));
    DDPPO_TRY(launch_fill(n.params + n.vis_b, Hd, 0.f, s));
  }
  DDPPO_TRY(unif(n.goal_w, 96, sqrtf(3.0f / 3.0f)));
  DDPPO_TRY(launch_fill(n.params + n.goal_b, 32, 0.f, s));
  DDPPO_TRY(unif(n.emb, 160, sqrtf(3.0f)));
  for (int l = 0; l < n.L; ++l) {
    LstmL& q = n.lstm[l];
    const float b = 1.0f / sqrtf((float)Hd);
    DDPPO_TRY(unif(q.wih, (int64_t)4 * Hd * q.In, b));
    DDPPO_TRY(unif(q.whh, (int64_t)4 * Hd * Hd, b));
    DDPPO_TRY(launch_fill(n.params + q.bih, 4 * Hd, 0.f, s));
    DDPPO_TRY(launch_fill(n.params + q.bhh, 4 * Hd, 0.f, s));
  }
  DDPPO_TRY(unif(n.actor_w, 4 * Hd, 0.01f * sqrtf(3.0f / Hd)));
  DDPPO_TRY(launch_fill(n.params + n.actor_b, 4, 0.f, s));
  DDPPO_TRY(unif(n.critic_w, Hd, sqrtf(3.0f / Hd)));
  DDPPO_TRY(launch_fill(n.params + n.critic_b, 1, 0.f, s));
  return DDPPO_OK;
}

// canonical fp32 params -> GEMM operands in the precision's dtype
int net_prep_weights(Net& n, cudaStream_t s) {
  for (ConvL* c : n.convs) {
    DDPPO_TRY(launch_conv_w_prep(n.params + c->w_off, c->cout, c->cin, c->k, c->Kp, c->wg, c->wgT,
                                 n.bf, s));
    if (c->dgrad_as_conv)
      DDPPO_TRY(launch_conv_w_flip(n.params + c->w_off, c->cout, c->cin, c->k, c->wgR, n.bf, s));
  }
  for (SxL& X : n.sx)
    DDPPO_TRY(launch_gconv_w_prep(n.params + X.c2.w_off, X.c2.C, X.c2.cpg, X.c2.wg, n.bf, s));
  if (n.f8) {
    // per-tensor E4M3 weights from the bf16 GEMM layout
    const int na = n.f8_act_slots;
    DDPPO_CHECK_CUDA(cudaMemsetAsync(n.f8_amax + na, 0, (size_t)(n.f8_slots - na) * 4, s));
    for (ConvL* c : n.convs) {
      if (!c->wg8) continue;
      const size_t cnt = (size_t)c->cout * c->Kp;
      DDPPO_TRY(launch_amax(c->wg, true, cnt, c->w8_amax, s));
      DDPPO_TRY(launch_quant_e4m3(c->wg, true, cnt, c->w8_amax, c->w8_scale, c->wg8, s));
    }
  }
  if (n.F > 0)
    DDPPO_TRY(launch_vis_w_prep(n.params + n.vis_w, n.H, n.featC, n.featHW, n.Wv, n.WvT, n.bf, s));
  for (int l = 0; l < n.L; ++l) {
    LstmL& q = n.lstm[l];
    const int G4 = 4 * n.H;
    DDPPO_TRY(launch_cast(n.params + q.wih, q.Wih, n.bf, (size_t)G4 * q.In, s));
    DDPPO_TRY(launch_transpose(n.params + q.wih, false, q.WihT, n.bf, G4, q.In, q.In, s));
    DDPPO_TRY(launch_cast(n.params + q.whh, q.Whh, n.bf, (size_t)G4 * n.H, s));
    DDPPO_TRY(launch_transpose(n.params + q.whh, false, q.WhhT, n.bf, G4, n.H, n.H, s));
    DDPPO_TRY(launch_add_vec(n.params + q.bih, n.params + q.bhh, q.bsum, G4, s));
  }
  return DDPPO_OK;
}

int net_create(ddppo_ctx* x) {
  Net* np = new Net();
  x->net = np;
  Net& n = *np;
  n.x = x;
  const ddppo_config& c = x->cfg;
  n.bf = c.precision >= 1;
  n.f8 = c.precision == 2;
  n.kind = c.net_kind;
  n.H = c.hidden;
  n.L = c.lstm_layers;
  n.E = c.num_envs;
  n.T = c.rollout_T;
  n.T_last = c.rollout_T;
  n.Emb = c.num_envs / c.minibatches;
  n.NS = std::max(n.T * n.Emb, n.E);
  // encoder pass size: the whole minibatch when it fits the automatic cap (8192 frames,
  // ~30 GB of activations for the 32-base ResNet), else chunks with recomputation
  // (the SE-ResNeXt keeps ~20 MB of activations per 128x128 frame: 1024 frames per pass)
  const int auto_chunk = c.net_kind >= 3 ? 1024 : 8192;
  n.NC = c.encoder_chunk > 0 ? std::min(c.encoder_chunk, n.NS) : std::min(n.NS, auto_chunk);
  n.NC = std::max(n.NC, n.E);  // an act step always fits one chunk
  n.NC = std::min(n.NC, n.NS);
  Layout lay;
  DDPPO_TRY(build_layout(n, lay));
  n.P = lay.off;
  n.pix = (size_t)n.inh * n.inw;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n.gws.num_sms, cudaDevAttrMultiProcessorCount, dev);
  n.gws.tc = &n.tc_count;
  n.gws.err = x->sb.err;
  DDPPO_TRY(nalloc(n, &n.params, n.P));
  DDPPO_TRY(nalloc(n, &n.grad, n.P));
  DDPPO_TRY(nalloc(n, &n.adam_m, n.P));
  DDPPO_TRY(nalloc(n, &n.adam_v, n.P));
  DDPPO_TRY(alloc_encoder(n));
  const size_t NS = n.NS, Hd = n.H, G4 = 4 * Hd;
  DDPPO_TRY(nalloc_op(n, &n.Wv, Hd * n.F));
  DDPPO_TRY(nalloc_op(n, &n.WvT, Hd * n.F));
  DDPPO_TRY(nalloc(n, &n.dWv, Hd * n.F));
  for (int l = 0; l < n.L; ++l) {
    LstmL& q = n.lstm[l];
    DDPPO_TRY(nalloc_op(n, &q.Wih, G4 * q.In));
    DDPPO_TRY(nalloc_op(n, &q.WihT, G4 * q.In));
    DDPPO_TRY(nalloc_op(n, &q.Whh, G4 * Hd));
    DDPPO_TRY(nalloc_op(n, &q.WhhT, G4 * Hd));
    DDPPO_TRY(nalloc(n, &q.bsum, G4));
    DDPPO_TRY(nalloc(n, &q.gates, NS * G4));
    DDPPO_TRY(nalloc(n, &q.c, NS * Hd));
    DDPPO_TRY(nalloc(n, &q.h, NS * Hd));
    DDPPO_TRY(nalloc_op(n, &q.hm, NS * Hd));
    DDPPO_TRY(nalloc_op(n, &q.y, NS * Hd));
  }
  DDPPO_TRY(nalloc_op(n, &n.featop, NS * n.F));
  DDPPO_TRY(nalloc(n, &n.dfeat, NS * n.F));
  DDPPO_TRY(nalloc_op(n, &n.featT, NS * n.F));
  DDPPO_TRY(nalloc_op(n, &n.x1, NS * n.In0));
  DDPPO_TRY(nalloc(n, &n.gx, NS * G4));
  DDPPO_TRY(nalloc(n, &n.gh, (size_t)n.E * G4));
  DDPPO_TRY(nalloc(n, &n.logits, NS * 4));
  DDPPO_TRY(nalloc(n, &n.values, NS));
  DDPPO_TRY(nalloc(n, &n.dh_top, NS * Hd));
  DDPPO_TRY(nalloc(n, &n.dX[0], NS * n.InMax));
  DDPPO_TRY(nalloc(n, &n.dX[1], NS * n.InMax));
  DDPPO_TRY(nalloc(n, &n.dg32, NS * G4));
  DDPPO_TRY(nalloc_op(n, &n.dgop, NS * G4));
  DDPPO_TRY(nalloc(n, &n.dh_rec, (size_t)n.E * Hd));
  DDPPO_TRY(nalloc(n, &n.dc_carry, (size_t)n.E * Hd));
  DDPPO_TRY(nalloc(n, &n.dv32, NS * Hd));
  DDPPO_TRY(nalloc_op(n, &n.dvop, NS * Hd));
  DDPPO_TRY(nalloc(n, &n.dlogits, NS * 4));
  DDPPO_TRY(nalloc(n, &n.dvalues, NS));
  n.scratch_elems = std::max((size_t)1 << 16, 5 * Hd * ((NS + 63) / 64) + 4096);
  DDPPO_TRY(nalloc(n, &n.scratch, n.scratch_elems));
  n.gws.partial_elems = (size_t)32 << 20;
  DDPPO_TRY(nalloc(n, &n.gws.partial, n.gws.partial_elems));
  if (n.bf) n.gws.tuner = tc_tuner_create((size_t)256 << 20);
  // minibatch
  const size_t NSmb = (size_t)n.T * n.Emb;
  DDPPO_TRY(nalloc_op(n, &n.obs_mb, NSmb * n.pix));
  DDPPO_TRY(nalloc(n, &n.goal_mb, NSmb * 3));
  DDPPO_TRY(nalloc(n, &n.preva_mb, NSmb));
  DDPPO_TRY(nalloc(n, &n.masks_mb, NSmb));
  DDPPO_TRY(nalloc(n, &n.act_mb, NSmb));
  DDPPO_TRY(nalloc(n, &n.logp_mb, NSmb));
  DDPPO_TRY(nalloc(n, &n.adv_mb, NSmb));
  DDPPO_TRY(nalloc(n, &n.ret_mb, NSmb));
  DDPPO_TRY(nalloc(n, &n.h0_mb, (size_t)n.L * n.Emb * Hd));
  DDPPO_TRY(nalloc(n, &n.c0_mb, (size_t)n.L * n.Emb * Hd));
  DDPPO_TRY(nalloc(n, &n.perm, n.E));
  DDPPO_TRY(nalloc(n, &n.adv_norm, (size_t)n.T * n.E));
  DDPPO_TRY(nalloc(n, &n.scal, 8));
  DDPPO_TRY(nalloc(n, &n.stats_tmp, 8 * 64));
  DDPPO_TRY(nalloc(n, &n.norm, 1));
  DDPPO_TRY(nalloc(n, &n.act_h, (size_t)n.L * n.E * Hd));
  DDPPO_TRY(nalloc(n, &n.act_c, (size_t)n.L * n.E * Hd));
  DDPPO_TRY(nalloc(n, &n.post_done, n.E));
  DDPPO_CHECK_CUDA(cudaMemset(n.adam_m, 0, n.P * 4));
  DDPPO_CHECK_CUDA(cudaMemset(n.adam_v, 0, n.P * 4));
  DDPPO_CHECK_CUDA(cudaMemset(n.stats_tmp, 0, 8 * 64 * 4));
  DDPPO_CHECK_CUDA(cudaStreamCreateWithFlags(&n.cap_stream, cudaStreamNonBlocking));
  DDPPO_TRY(nalloc(n, &n.d_steps, 2));
  DDPPO_TRY(nalloc(n, &n.lstm_bar, 4));
  DDPPO_CHECK_CUDA(cudaMemset(n.d_steps, 0, 2 * sizeof(int64_t)));
  DDPPO_CHECK_CUDA(cudaEventCreateWithFlags(&n.ev_a, cudaEventDisableTiming));
  DDPPO_CHECK_CUDA(cudaEventCreateWithFlags(&n.ev_b, cudaEventDisableTiming));
  for (int i = 0; i < 2 * 4096; ++i) {
    DDPPO_CHECK_CUDA(cudaEventCreate(&n.timer.ev[i]));
    DDPPO_CHECK_CUDA(cudaEventCreate(&n.rc_timer.ev[i]));
  }
  DDPPO_TRY(init_params(n, 0));
  DDPPO_TRY(net_prep_weights(n, 0));
  return DDPPO_OK;
}

void net_destroy(ddppo_ctx* x) {
  if (!x || !x->net) return;
  Net& n = *x->net;
  tc_tuner_destroy(n.gws.tuner);
  for (void* p : n.allocs) cudaFree(p);
  if (n.graph_exec) cudaGraphExecDestroy(n.graph_exec);
  if (n.upd_exec) cudaGraphExecDestroy(n.upd_exec);
  if (n.cap_stream) cudaStreamDestroy(n.cap_stream);
  if (n.ev_a) cudaEventDestroy(n.ev_a);
  if (n.ev_b) cudaEventDestroy(n.ev_b);
  for (int i = 0; i < 2 * 4096; ++i) {
    if (n.timer.ev[i]) cudaEventDestroy(n.timer.ev[i]);
    if (n.rc_timer.ev[i]) cudaEventDestroy(n.rc_timer.ev[i]);
  }
  delete x->net;
  x->net = nullptr;
}

// ---------------------------------------------------------------- encoder
static int G(Net& n, const GemmDesc& d, cudaStream_t s) { return gemm(d, n.bf, n.gws, s, &n.timer); }

static ConvShape conv_shape(const ConvL& c, int N) {
  ConvShape cs;
  cs.N = N; cs.H = c.H; cs.W = c.W; cs.C = c.cin; cs.Ho = c.Ho; cs.Wo = c.Wo;
  cs.k = c.k; cs.s = c.s; cs.p = c.p;
  cs.Cout = c.cout;
  return cs;
}

// forward convolution. in_bf (bf16 NHWC copy of the input, BF16 form) lets the tensor-core
// GEMM gather the patches itself; otherwise im2col materialises them first
static int conv_fwd(Net& n, ConvL& c, const void* in, bool in_bf16, int N, float* out, bool bias_relu,
                    cudaStream_t s, const __nv_bfloat16* in_bf = nullptr,
                    const uint8_t* in_f8 = nullptr, const float* in_scale = nullptr) {
  GemmDesc d;
  d.M = N * c.Ho * c.Wo; d.N = c.cout; d.K = c.Kp;
  d.B = c.wg; d.ldb = c.Kp;
  d.C = out; d.ldc = c.cout;
  if (bias_relu) { d.bias = n.params + c.b_off; d.relu = 1; }
  const ConvShape cs = conv_shape(c, N);
  if (in_f8 && c.wg8) {
    // FP8 inference: E4M3 input and weights, the product rescaled in the epilogue
    d.conv = &cs;
    d.fp8 = 1;
    d.A = in_f8; d.lda = d.K;
    d.B = c.wg8;
    d.scale_a = in_scale; d.scale_b = c.w8_scale;
    return G(n, d, s);
  }
  if (n.bf && in_bf && c.Kp == c.k * c.k * c.cin && gemm_conv_supported(cs, in_bf)) {
    d.conv = &cs;
    d.A = in_bf; d.lda = d.K;
    return G(n, d, s);
  }
  const ConvGeom g = geom(c, N);
  DDPPO_TRY(launch_im2col(g, in, in_bf16, n.col, n.bf, false, s));
  d.A = n.col; d.lda = c.Kp;
  return G(n, d, s);
}

// weight gradient (accumulated over chunks) and, if dx, the input gradient.
//   dW[co, kk] += sum_m dz[m, co] col[m, kk]   (both operands read as stored: MN-major)
//   dcol[m, kk] = sum_co dz[m, co] W[co, kk]   then col2im
static int conv_bwd(Net& n, ConvL& c, const void* in, bool in_bf16, int N, const void* dzop,
                    float* dx, bool dx_acc, bool first, cudaStream_t s,
                    const __nv_bfloat16* in_bf = nullptr) {
  const ConvGeom g = geom(c, N);
  const int M = N * c.Ho * c.Wo;
  GemmDesc w;
  w.M = c.cout; w.N = c.Kp; w.K = M;
  w.A = dzop; w.lda = c.cout; w.a_t = 1;
  w.C = c.dwg; w.ldc = c.Kp; w.beta = first ? 0.f : 1.f;
  const ConvShape cs = conv_shape(c, N);
  const void* x_bf = in_bf ? (const void*)in_bf : (in_bf16 ? in : nullptr);
  if (n.bf && x_bf && c.Kp == c.k * c.k * c.cin && c.cout % 8 == 0 &&
      (conv_wgrad_halo_ok(cs, x_bf, dzop) || gemm_convw_supported(cs, x_bf, dzop))) {
    w.convw = &cs;  // the GEMM gathers the shifted input rows itself
    w.B = x_bf;
  } else {
    if (in_bf) DDPPO_TRY(launch_im2col(g, in_bf, true, n.col, n.bf, false, s));
    else DDPPO_TRY(launch_im2col(g, in, in_bf16, n.col, n.bf, false, s));
    w.B = n.col; w.ldb = c.Kp; w.b_t = 1;
  }
  DDPPO_TRY(G(n, w, s));
  if (dx && c.dgrad_as_conv) {
    // dx = conv(dz, flipped kernel): im2col of dz (C = cout) then one GEMM into dx
    ConvGeom gd;
    gd.N = N; gd.H = c.Ho; gd.W = c.Wo; gd.C = c.cout; gd.Ho = c.H; gd.Wo = c.W; gd.Cout = c.cin;
    gd.k = c.k; gd.s = 1; gd.p = c.p; gd.K = c.k * c.k * c.cout; gd.Kp = gd.K;
    GemmDesc d;
    d.M = N * c.H * c.W; d.N = c.cin; d.K = gd.K;
    d.B = c.wgR; d.ldb = gd.K;
    d.C = dx; d.ldc = c.cin; d.beta = dx_acc ? 1.f : 0.f;
    ConvShape cs;
    cs.N = N; cs.H = c.Ho; cs.W = c.Wo; cs.C = c.cout; cs.Ho = c.H; cs.Wo = c.W;
    cs.k = c.k; cs.s = 1; cs.p = c.p; cs.Cout = c.cin;
    if (n.bf && gemm_conv_supported(cs, dzop)) {
      d.conv = &cs;  // the output gradient (bf16 NHWC) is gathered by the GEMM itself
      d.A = dzop; d.lda = d.K;
    } else {
      DDPPO_TRY(launch_im2col(gd, dzop, n.bf, n.col, n.bf, false, s));
      d.A = n.col; d.lda = gd.K;
    }
    DDPPO_TRY(G(n, d, s));
  } else if (dx) {
    GemmDesc d;
    d.M = M; d.N = c.Kp; d.K = c.cout;
    d.A = dzop; d.lda = c.cout; d.B = c.wgT; d.ldb = c.cout;
    d.C = n.dcol; d.ldc = c.Kp;
    DDPPO_TRY(G(n, d, s));
    DDPPO_TRY(launch_col2im(g, n.dcol, dx, dx_acc, s));
  }
  return DDPPO_OK;
}

static int gn_fwd(Net& n, GNL& g, const float* z, int N, int HW, float* out, bool relu,
                  const float* resid, const GNL* gd, const float* zd, cudaStream_t s,
                  __nv_bfloat16* out_bf = nullptr, uint8_t* out_f8 = nullptr, int f8_slot = -1) {
  const float eps = 1e-5f;
  GNApply a{};
  a.z = z; a.mean = g.mean; a.rstd = g.rstd;
  a.gamma = n.params + g.g_off; a.beta = n.params + g.b_off;
  a.resid = resid;
  if (gd) {
    a.zd = zd; a.mean_d = gd->mean; a.rstd_d = gd->rstd;
    a.gamma_d = n.params + gd->g_off; a.beta_d = n.params + gd->b_off;
  }
  a.out = out;
  a.out_bf = out_bf;
  if (out_f8) {
    a.out_f8 = out_f8;
    a.f8_scale = n.f8_scale + f8_slot;
    a.f8_amax = n.f8_amax + f8_slot;
  }
  a.relu = relu ? 1 : 0;
  if (n.gn_fused_on) {
    // statistics and normalisation in one launch when the grid fits one resident wave
    bool done = false;
    DDPPO_TRY(launch_gn_fused(a, N, HW, g.C, eps, n.gnw, n.gws.err, s, &done));
    if (done) return DDPPO_OK;
  }
  DDPPO_TRY(launch_gn_stats(z, N, HW, g.C, eps, g.mean, g.rstd, n.gnw, s));
  if (gd) DDPPO_TRY(launch_gn_stats(zd, N, HW, gd->C, eps, gd->mean, gd->rstd, n.gnw, s));
  return launch_gn_apply(a, N, HW, g.C, s);
}

// GroupNorm backward into n.dzop (op dtype). relu_y: the output of the ReLU that followed
// the normalisation (its mask is applied to dy here); g_out receives the masked gradient.
static int gn_bwd(Net& n, GNL& g, const float* dy, const float* z, int N, int HW, bool first,
                  cudaStream_t s, const float* relu_y = nullptr, float* g_out = nullptr) {
  GNBack b{};
  b.dy = dy; b.relu_y = relu_y; b.g_out = g_out;
  b.z = z; b.mean = g.mean; b.rstd = g.rstd; b.gamma = n.params + g.g_off;
  b.m1 = n.gn_m1; b.m2 = n.gn_m2;
  b.dzop = n.dzop; b.op_bf16 = n.bf;
  b.dgamma_part = n.gnp_g; b.dbeta_part = n.gnp_b;
  DDPPO_TRY(launch_gn_bwd(b, N, HW, g.C, n.gnw, s));
  DDPPO_TRY(launch_colsum2(n.gnp_g, n.gnp_b, N, g.C, g.C, n.grad + g.g_off, n.grad + g.b_off,
                           !first, s));
  return DDPPO_OK;
}

static GConv gconv_of(const GConvL& g, int N) {
  GConv c;
  c.N = N; c.H = g.H; c.W = g.W; c.C = g.C; c.cpg = g.cpg; c.s = g.s; c.Ho = g.Ho; c.Wo = g.Wo;
  return c;
}

static SeArgs se_args(Net& n, SxL& X, int N) {
  SeArgs e{};
  e.N = N; e.HW = X.HW; e.C = X.C; e.Cr = X.Cr;
  e.u = X.u;
  e.W1 = n.params + X.se1_w; e.b1 = n.params + X.se1_b;
  e.W2 = n.params + X.se2_w; e.b2 = n.params + X.se2_b;
  e.m = X.m; e.a = X.a; e.gate = X.gate;
  e.y = X.y; e.y_bf = n.bf ? X.y_bf : nullptr;
  e.dg = n.se_dg; e.dq = n.se_dq; e.dh = n.se_dh; e.dm = n.se_dm;
  e.gW1 = n.grad + X.se1_w; e.gb1 = n.grad + X.se1_b;
  e.gW2 = n.grad + X.se2_w; e.gb2 = n.grad + X.se2_b;
  return e;
}

// SE-ResNeXt bottleneck forward: x (fp32) and its bf16 copy (BF16 form) -> X.y (+ X.y_bf)
static int sx_block_fwd(Net& n, SxL& X, int N, const float* x, const __nv_bfloat16* x_bf,
                        cudaStream_t s) {
  const int HWi = X.c1.H * X.c1.W;
  DDPPO_TRY(conv_fwd(n, X.c1, x, false, N, X.c1.z, false, s, x_bf));
  DDPPO_TRY(gn_fwd(n, X.n1, X.c1.z, N, HWi, X.n1.out, true, nullptr, nullptr, nullptr, s,
                   X.n1.out_bf));
  const void* g_in = n.bf ? (const void*)X.n1.out_bf : (const void*)X.n1.out;
  DDPPO_TRY(launch_gconv_fwd(gconv_of(X.c2, N), g_in, X.c2.wg, X.c2.z, n.bf, s));
  DDPPO_TRY(gn_fwd(n, X.n2, X.c2.z, N, X.HW, X.n2.out, true, nullptr, nullptr, nullptr, s,
                   X.n2.out_bf));
  DDPPO_TRY(conv_fwd(n, X.c3, X.n2.out, false, N, X.c3.z, false, s, X.n2.out_bf));
  DDPPO_TRY(gn_fwd(n, X.n3, X.c3.z, N, X.HW, X.u, false, nullptr, nullptr, nullptr, s));
  const float* sc = x;
  if (X.down) {
    DDPPO_TRY(conv_fwd(n, X.d, x, false, N, X.d.z, false, s, x_bf));
    DDPPO_TRY(gn_fwd(n, X.nd, X.d.z, N, X.HW, X.sc, false, nullptr, nullptr, nullptr, s));
    sc = X.sc;
  }
  SeArgs e = se_args(n, X, N);
  e.sc = sc;
  return launch_se_fwd(e, s);
}

// its backward: gcur holds the gradient of X.y and receives that of the block input x;
// gA, gB are scratch of the same size (the three buffers may be rotated: gcur is updated)
static int sx_block_bwd(Net& n, SxL& X, int N, const float* x, const __nv_bfloat16* x_bf,
                        bool first, float*& gcur, float*& gA, float*& gB, cudaStream_t s) {
  const int HWi = X.c1.H * X.c1.W;
  SeArgs e = se_args(n, X, N);
  // gcur <- gradient through the output ReLU (the shortcut's); gA <- the branch's (du)
  DDPPO_TRY(launch_se_bwd(e, gcur, gcur, gA, !first, s));
  DDPPO_TRY(gn_bwd(n, X.n3, gA, X.c3.z, N, X.HW, first, s));
  DDPPO_TRY(conv_bwd(n, X.c3, X.n2.out, false, N, n.dzop, gB, false, first, s, X.n2.out_bf));
  DDPPO_TRY(gn_bwd(n, X.n2, gB, X.c2.z, N, X.HW, first, s, X.n2.out));
  const GConv gc = gconv_of(X.c2, N);
  const void* g_in = n.bf ? (const void*)X.n1.out_bf : (const void*)X.n1.out;
  DDPPO_TRY(launch_gconv_wgrad(gc, g_in, n.dzop, n.gw_part, n.gw_part_elems, n.gws.num_sms,
                               n.grad + X.c2.w_off, first ? 0.f : 1.f, n.bf, s));
  DDPPO_TRY(launch_gconv_dgrad(gc, n.dzop, X.c2.wg, gA, false, n.bf, s));
  DDPPO_TRY(gn_bwd(n, X.n1, gA, X.c1.z, N, HWi, first, s, X.n1.out));
  if (X.down) {
    DDPPO_TRY(conv_bwd(n, X.c1, x, false, N, n.dzop, gB, false, first, s, x_bf));
    DDPPO_TRY(gn_bwd(n, X.nd, gcur, X.d.z, N, X.HW, first, s));
    DDPPO_TRY(conv_bwd(n, X.d, x, false, N, n.dzop, gB, true, first, s, x_bf));
    float* t = gcur; gcur = gB; gB = t;
  } else {
    DDPPO_TRY(conv_bwd(n, X.c1, x, false, N, n.dzop, gcur, true, first, s, x_bf));
  }
  return DDPPO_OK;
}

// forward of one chunk of N images: obs (op dtype) -> featop rows (op dtype). f8: the
// act-time pass of FP8 inference (N <= E): every convolution after the stem reads E4M3
// copies of its input and weights; the activation scales advance once per pass
static int encoder_fwd(Net& n, const void* obs, int N, void* featop_rows, cudaStream_t s,
                       bool f8 = false) {
  if (n.kind == 0) {
    DDPPO_TRY(conv_fwd(n, n.nat[0], obs, n.bf, N, n.nat[0].z, true, s));
    DDPPO_TRY(conv_fwd(n, n.nat[1], n.nat[0].z, false, N, n.nat[1].z, true, s));
    DDPPO_TRY(conv_fwd(n, n.nat[2], n.nat[1].z, false, N, n.nat[2].z, true, s));
    return launch_cast(n.nat[2].z, featop_rows, n.bf, (size_t)N * n.F, s);
  }
  ConvL& st = n.stem;
  DDPPO_TRY(conv_fwd(n, st, obs, n.bf, N, st.z, false, s));
  if (st.cout % 4 == 0) {
    // GroupNorm + ReLU + max pool in one pass: the full-resolution activation is never
    // stored (the backward recomputes its ReLU mask from z)
    DDPPO_TRY(launch_gn_stats(st.z, N, st.Ho * st.Wo, st.cout, 1e-5f, n.stem_n.mean, n.stem_n.rstd,
                              n.gnw, s));
    GNApply a{};
    a.z = st.z; a.mean = n.stem_n.mean; a.rstd = n.stem_n.rstd;
    a.gamma = n.params + n.stem_n.g_off; a.beta = n.params + n.stem_n.b_off;
    a.relu = 1;
    if (f8) {
      a.out_f8 = n.pool_f8;
      a.f8_scale = n.f8_scale + n.pool_slot;
      a.f8_amax = n.f8_amax + n.pool_slot;
    }
    DDPPO_TRY(launch_gn_relu_maxpool(a, N, st.Ho, st.Wo, st.cout, n.pool, f8 ? nullptr : n.pool_bf,
                                     n.pool_arg, s));
  } else {
    DDPPO_TRY(gn_fwd(n, n.stem_n, st.z, N, st.Ho * st.Wo, n.stem_n.out, true, nullptr, nullptr,
                     nullptr, s));
    DDPPO_TRY(launch_maxpool_fwd(n.stem_n.out, N, st.Ho, st.Wo, st.cout, n.pool, n.pool_arg,
                                 n.pool_bf, s));
  }
  const float* cur = n.pool;
  const __nv_bfloat16* cur_bf = f8 ? nullptr : n.pool_bf;
  if (!n.sx.empty()) {
    for (SxL& X : n.sx) {
      DDPPO_TRY(sx_block_fwd(n, X, N, cur, cur_bf, s));
      cur = X.y;
      cur_bf = n.bf ? X.y_bf : nullptr;
    }
    const SxL& L = n.sx.back();
    DDPPO_TRY(conv_fwd(n, n.cmp, L.y, false, N, n.cmp.z, false, s, L.y_bf));
    DDPPO_TRY(gn_fwd(n, n.cmp_n, n.cmp.z, N, n.featHW, n.cmp_n.out, true, nullptr, nullptr, nullptr, s));
    return launch_cast(n.cmp_n.out, featop_rows, n.bf, (size_t)N * n.F, s);
  }
  const uint8_t* cur_f8 = f8 ? n.pool_f8 : nullptr;
  const float* cur_sc = f8 ? n.f8_scale + n.pool_slot : nullptr;
  for (auto& B : n.blocks) {
    const int HW = B.c1.Ho * B.c1.Wo;
    DDPPO_TRY(conv_fwd(n, B.c1, cur, false, N, B.c1.z, false, s, cur_bf, cur_f8, cur_sc));
    DDPPO_TRY(gn_fwd(n, B.n1, B.c1.z, N, HW, B.n1.out, true, nullptr, nullptr, nullptr, s,
                     f8 ? nullptr : B.n1.out_bf, f8 ? B.n1.out_f8 : nullptr, B.n1.f8_slot));
    DDPPO_TRY(conv_fwd(n, B.c2, B.n1.out, false, N, B.c2.z, false, s, f8 ? nullptr : B.n1.out_bf,
                       f8 ? B.n1.out_f8 : nullptr, f8 ? n.f8_scale + B.n1.f8_slot : nullptr));
    uint8_t* y_f8 = f8 ? B.y_f8 : nullptr;
    __nv_bfloat16* y_bf = f8 ? nullptr : B.y_bf;
    if (B.down) {
      DDPPO_TRY(conv_fwd(n, B.d, cur, false, N, B.d.z, false, s, cur_bf, cur_f8, cur_sc));
      DDPPO_TRY(gn_fwd(n, B.n2, B.c2.z, N, HW, B.y, true, nullptr, &B.nd, B.d.z, s, y_bf, y_f8,
                       B.y_slot));
    } else {
      DDPPO_TRY(gn_fwd(n, B.n2, B.c2.z, N, HW, B.y, true, cur, nullptr, nullptr, s, y_bf, y_f8,
                       B.y_slot));
    }
    cur = B.y;
    cur_bf = y_bf;
    cur_f8 = y_f8;
    cur_sc = f8 ? n.f8_scale + B.y_slot : nullptr;
  }
  DDPPO_TRY(conv_fwd(n, n.cmp, cur, false, N, n.cmp.z, false, s, cur_bf, cur_f8, cur_sc));
  DDPPO_TRY(gn_fwd(n, n.cmp_n, n.cmp.z, N, n.featHW, n.cmp_n.out, true, nullptr, nullptr, nullptr, s));
  if (f8) DDPPO_TRY(launch_f8_scale_update(n.f8_scale, n.f8_amax, n.f8_act_slots, s));
  return launch_cast(n.cmp_n.out, featop_rows, n.bf, (size_t)N * n.F, s);
}

// backward of one chunk: dfeat rows (fp32, NHWC-flattened) -> weight grads
static int encoder_bwd(Net& n, const void* obs, int N, const float* dfeat_rows, bool first,
                       cudaStream_t s) {
  if (n.kind == 0) {
    ConvL* c = n.nat;
    float* gbuf[3] = {n.g0, n.g1, n.g2};
    const float* dy = dfeat_rows;
    for (int i = 2; i >= 0; --i) {
      const size_t cnt = (size_t)N * c[i].Ho * c[i].Wo * c[i].cout;
      DDPPO_TRY(launch_relu_bwd(dy, c[i].z, cnt, gbuf[i], n.dzop, n.bf, s));
      DDPPO_TRY(launch_colsum(gbuf[i], N * c[i].Ho * c[i].Wo, c[i].cout, c[i].cout,
                              n.grad + c[i].b_off, !first, s));
      const void* in = i == 0 ? obs : (const void*)c[i - 1].z;
      float* dx = i == 0 ? nullptr : gbuf[i - 1];
      DDPPO_TRY(conv_bwd(n, c[i], in, i == 0 ? n.bf : false, N, n.dzop, dx, false, first, s));
      dy = dx;
    }
    return DDPPO_OK;
  }
  // compression conv
  DDPPO_TRY(gn_bwd(n, n.cmp_n, dfeat_rows, n.cmp.z, N, n.featHW, first, s, n.cmp_n.out));
  const float* last_y = n.sx.empty() ? n.blocks[7].y : n.sx.back().y;
  const __nv_bfloat16* last_bf = n.sx.empty() ? n.blocks[7].y_bf : n.sx.back().y_bf;
  DDPPO_TRY(conv_bwd(n, n.cmp, last_y, false, N, n.dzop, n.g1, false, first, s, last_bf));
  // residual blocks, last to first. gcur: gradient of the block output (before its ReLU)
  float* gcur = n.g1;
  float* gA = n.g0;
  float* gB = n.g2;
  for (int bi = (int)n.sx.size() - 1; bi >= 0; --bi) {
    const float* xin = bi > 0 ? n.sx[bi - 1].y : n.pool;
    const __nv_bfloat16* xin_bf = bi > 0 ? n.sx[bi - 1].y_bf : n.pool_bf;
    DDPPO_TRY(sx_block_bwd(n, n.sx[bi], N, xin, xin_bf, first, gcur, gA, gB, s));
  }
  for (int bi = n.sx.empty() ? 7 : -1; bi >= 0; --bi) {
    BlockL& B = n.blocks[bi];
    const int HW = B.c1.Ho * B.c1.Wo;
    const float* xin = bi > 0 ? n.blocks[bi - 1].y : n.pool;
    const __nv_bfloat16* xin_bf = bi > 0 ? n.blocks[bi - 1].y_bf : n.pool_bf;
    // the ReLU after the sum masks gcur; with an identity skip the masked gradient is
    // kept (written back in place) and the first conv's input gradient accumulates onto it
    DDPPO_TRY(gn_bwd(n, B.n2, gcur, B.c2.z, N, HW, first, s, B.y, B.down ? nullptr : gcur));
    DDPPO_TRY(conv_bwd(n, B.c2, B.n1.out, false, N, n.dzop, gA, false, first, s, B.n1.out_bf));
    DDPPO_TRY(gn_bwd(n, B.n1, gA, B.c1.z, N, HW, first, s, B.n1.out));
    if (B.down) {
      DDPPO_TRY(conv_bwd(n, B.c1, xin, false, N, n.dzop, gB, false, first, s, xin_bf));
      DDPPO_TRY(gn_bwd(n, B.nd, gcur, B.d.z, N, HW, first, s, B.y));
      DDPPO_TRY(conv_bwd(n, B.d, xin, false, N, n.dzop, gB, true, first, s, xin_bf));
      float* t = gcur; gcur = gB; gB = t;
    } else {
      DDPPO_TRY(conv_bwd(n, B.c1, xin, false, N, n.dzop, gcur, true, first, s, xin_bf));
    }
  }
  // max pool, stem GN + ReLU, stem conv (no input gradient)
  ConvL& st = n.stem;
  if (st.cout % 4 == 0) {
    // the max-pool gradient scattered once; the GroupNorm backward recomputes the ReLU
    // mask from z (the full-resolution activation was never stored)
    DDPPO_TRY(launch_maxpool_bwd(gcur, n.pool_arg, N, st.Ho, st.Wo, st.cout, gA, s));
    GNBack b{};
    b.dy = gA;
    b.z = st.z; b.mean = n.stem_n.mean; b.rstd = n.stem_n.rstd;
    b.gamma = n.params + n.stem_n.g_off; b.beta = n.params + n.stem_n.b_off;
    b.relu_from_z = 1;
    b.m1 = n.gn_m1; b.m2 = n.gn_m2;
    b.dzop = n.dzop; b.op_bf16 = n.bf;
    b.dgamma_part = n.gnp_g; b.dbeta_part = n.gnp_b;
    DDPPO_TRY(launch_gn_bwd(b, N, st.Ho * st.Wo, st.cout, n.gnw, s));
    DDPPO_TRY(launch_colsum2(n.gnp_g, n.gnp_b, N, st.cout, st.cout, n.grad + n.stem_n.g_off,
                             n.grad + n.stem_n.b_off, !first, s));
  } else {
    DDPPO_TRY(launch_maxpool_bwd(gcur, n.pool_arg, N, st.Ho, st.Wo, st.cout, gA, s));
    DDPPO_TRY(gn_bwd(n, n.stem_n, gA, st.z, N, st.Ho * st.Wo, first, s, n.stem_n.out));
  }
  DDPPO_TRY(conv_bwd(n, st, obs, n.bf, N, n.dzop, nullptr, false, first, s));
  return DDPPO_OK;
}

// ---------------------------------------------------------------- forward / backward
// the LSTM layers over a [T, E] segment: layer 0 reads n.x1 (op dtype, [N, In0]); every
// step's gates, cell and hidden state stay in the layer buffers for the backward
static int lstm_forward(Net& n, int T, int E, const uint8_t* masks, const float* h0,
                        const float* c0, cudaStream_t s) {
  const int N = T * E, Hd = n.H, G4 = 4 * Hd;
  const bool seq = n.lstm_mode == 1 && lstm_seq_supported(Hd, E, n.gws.num_sms);
  // (a single step -- the act path -- gains nothing from the resident weights: step path)
  const bool tc = n.lstm_mode == 2 && n.bf && T > 1 && lstm_tc_supported(Hd, E, n.gws.num_sms);
  for (int l = 0; l < n.L; ++l) {
    LstmL& q = n.lstm[l];
    GemmDesc gx;
    gx.M = N; gx.N = G4; gx.K = q.In;
    gx.A = l == 0 ? n.x1 : n.lstm[l - 1].y; gx.lda = l == 0 ? n.In0 : Hd;
    gx.B = q.Wih; gx.ldb = q.In;
    gx.C = n.gx; gx.ldc = G4; gx.bias = q.bsum;
    DDPPO_TRY(G(n, gx, s));
    if (seq) {
      // the whole recurrence of the layer in one launch
      LstmSeq a{};
      a.T = T; a.E = E; a.H = Hd;
      a.gx = n.gx; a.m = masks; a.h0 = h0 + (size_t)l * E * Hd; a.c0 = c0 + (size_t)l * E * Hd;
      a.Whh = q.Whh;
      a.gates = q.gates; a.c = q.c; a.h = q.h; a.y_op = q.y; a.hm = q.hm;
      a.bar = n.lstm_bar; a.err = n.gws.err; a.op_bf16 = n.bf ? 1 : 0;
      DDPPO_TRY(launch_lstm_seq_fwd(a, n.gws.num_sms, s));
      continue;
    }
    if (tc) {
      DDPPO_TRY(launch_mask_state(h0 + (size_t)l * E * Hd, masks, E, Hd, q.hm, true, s));
      LstmTc a{};
      a.T = T; a.E = E; a.H = Hd;
      a.gx = n.gx; a.m = masks; a.c0 = c0 + (size_t)l * E * Hd;
      a.Whh = (const __nv_bfloat16*)q.Whh;
      a.gates = q.gates; a.c = q.c; a.h = q.h;
      a.y_op = (__nv_bfloat16*)q.y; a.hm = (__nv_bfloat16*)q.hm;
      a.bar = n.lstm_bar; a.err = n.gws.err;
      DDPPO_TRY(launch_lstm_tc_fwd(a, n.gws.num_sms, s));
      continue;
    }
    DDPPO_TRY(launch_mask_state(h0 + (size_t)l * E * Hd, masks, E, Hd, q.hm, n.bf, s));
    for (int t = 0; t < T; ++t) {
      GemmDesc gh;
      gh.M = E; gh.N = G4; gh.K = Hd;
      gh.A = opoff(n, q.hm, (size_t)t * E * Hd); gh.lda = Hd;
      gh.B = q.Whh; gh.ldb = Hd;
      gh.C = n.gh; gh.ldc = G4;
      DDPPO_TRY(G(n, gh, s));
      LstmStep st;
      st.E = E; st.H = Hd;
      st.gx = n.gx + (size_t)t * E * G4;
      st.gh = n.gh;
      st.c_prev = t == 0 ? c0 + (size_t)l * E * Hd : q.c + (size_t)(t - 1) * E * Hd;
      st.m = masks + (size_t)t * E;
      st.m_next = t + 1 < T ? masks + (size_t)(t + 1) * E : nullptr;
      st.gates = q.gates + (size_t)t * E * G4;
      st.c = q.c + (size_t)t * E * Hd;
      st.h = q.h + (size_t)t * E * Hd;
      st.y_op = opoff(n, q.y, (size_t)t * E * Hd);
      st.hm_next = t + 1 < T ? opoff(n, q.hm, (size_t)(t + 1) * E * Hd) : nullptr;
      st.op_bf16 = n.bf;
      DDPPO_TRY(launch_lstm_fwd(st, s));
    }
  }
  return DDPPO_OK;
}

// back-propagation through time over the last [T, E] forward of the LSTM layers: dtop
// [N, H] is the gradient of the top layer's outputs; accumulates the LSTM parameter
// gradients into n.grad and leaves the gradient of layer 0's input ([N, In0], fp32) in
// *dx0
static int lstm_backward(Net& n, int T, int E, const uint8_t* masks, const float* c0,
                         const float* dtop, const float** dx0, cudaStream_t s) {
  const int N = T * E, Hd = n.H, G4 = 4 * Hd;
  const bool seq = n.lstm_mode == 1 && lstm_seq_supported(Hd, E, n.gws.num_sms);
  const float* dabove = dtop;
  for (int l = n.L - 1; l >= 0; --l) {
    LstmL& q = n.lstm[l];
    if (seq) {
      LstmSeq a{};
      a.T = T; a.E = E; a.H = Hd;
      a.m = masks; a.c0 = c0 + (size_t)l * E * Hd; a.Whh = q.Whh;
      a.gates = q.gates; a.c = q.c;
      a.dh_above = dabove; a.dg32 = n.dg32; a.dg_op = n.dgop;
      a.bar = n.lstm_bar; a.err = n.gws.err; a.op_bf16 = n.bf ? 1 : 0;
      DDPPO_TRY(launch_lstm_seq_bwd(a, n.gws.num_sms, s));
    }
    if (!seq) DDPPO_CHECK_CUDA(cudaMemsetAsync(n.dc_carry, 0, (size_t)E * Hd * sizeof(float), s));
    for (int t = seq ? -1 : T - 1; t >= 0; --t) {
      LstmBack b;
      b.E = E; b.H = Hd;
      b.gates = q.gates + (size_t)t * E * G4;
      b.c = q.c + (size_t)t * E * Hd;
      b.c_prev = t == 0 ? c0 + (size_t)l * E * Hd : q.c + (size_t)(t - 1) * E * Hd;
      b.m = masks + (size_t)t * E;
      b.m_next = t + 1 < T ? masks + (size_t)(t + 1) * E : nullptr;
      b.dh_above = dabove + (size_t)t * E * Hd;
      b.dh_rec = t + 1 < T ? n.dh_rec : nullptr;
      b.dc_carry = n.dc_carry;
      b.dg32 = n.dg32 + (size_t)t * E * G4;
      b.dg_op = opoff(n, n.dgop, (size_t)t * E * G4);
      b.op_bf16 = n.bf;
      DDPPO_TRY(launch_lstm_bwd(b, s));
      if (t > 0) {
        GemmDesc r;
        r.M = E; r.N = Hd; r.K = G4;
        r.A = opoff(n, n.dgop, (size_t)t * E * G4); r.lda = G4;
        r.B = q.WhhT; r.ldb = G4;
        r.C = n.dh_rec; r.ldc = Hd;
        DDPPO_TRY(G(n, r, s));
      }
    }
    float* dX = n.dX[l & 1];
    GemmDesc dx;
    dx.M = N; dx.N = q.In; dx.K = G4;
    dx.A = n.dgop; dx.lda = G4; dx.B = q.WihT; dx.ldb = G4;
    dx.C = dX; dx.ldc = q.In;
    DDPPO_TRY(G(n, dx, s));
    const void* X = l == 0 ? n.x1 : n.lstm[l - 1].y;
    const int ldX = l == 0 ? n.In0 : Hd;
    // dW_ih[g, i] = sum_n dG[n, g] X[n, i]; dW_hh[g, j] = sum_n dG[n, g] Hm[n, j]
    GemmDesc wi;
    wi.M = G4; wi.N = q.In; wi.K = N;
    wi.A = n.dgop; wi.lda = G4; wi.a_t = 1; wi.B = X; wi.ldb = ldX; wi.b_t = 1;
    wi.C = n.grad + q.wih; wi.ldc = q.In;
    DDPPO_TRY(G(n, wi, s));
    GemmDesc wh;
    wh.M = G4; wh.N = Hd; wh.K = N;
    wh.A = n.dgop; wh.lda = G4; wh.a_t = 1; wh.B = q.hm; wh.ldb = Hd; wh.b_t = 1;
    wh.C = n.grad + q.whh; wh.ldc = Hd;
    DDPPO_TRY(G(n, wh, s));
    DDPPO_TRY(launch_colsum2(n.dg32, n.dg32, N, G4, G4, n.grad + q.bih, n.grad + q.bhh, false, s));
    dabove = dX;
  }
  *dx0 = dabove;
  return DDPPO_OK;
}

// encoder backward over N frames of obs given n.dfeat (NHWC-flattened feature rows, fp32):
// last chunk first (its activations are still resident), the others recomputed; the
// convolution weight gradients land in n.grad
static int encoder_backward(Net& n, const void* obs, int N, cudaStream_t s) {
  const int nch = (N + n.NC - 1) / n.NC;
  for (int c = nch - 1; c >= 0; --c) {
    const int r0 = c * n.NC, rn = std::min(n.NC, N - r0);
    const void* obs_c = opoff(n, obs, (size_t)r0 * n.pix);
    if (c != n.ev_valid_chunk) {
      DDPPO_TRY(encoder_fwd(n, obs_c, rn, n.featT, s));  // feature rows are not needed again
      n.ev_valid_chunk = c;
    }
    DDPPO_TRY(encoder_bwd(n, obs_c, rn, n.dfeat + (size_t)r0 * n.F, c == nch - 1, s));
  }
  for (ConvL* c : n.convs)
    DDPPO_TRY(launch_conv_w_grad(c->dwg, c->cout, c->cin, c->k, c->Kp, n.grad + c->w_off, s));
  return DDPPO_OK;
}

int net_forward(Net& n, int T, int E, const void* obs, const float* goal, const int32_t* prev_a,
                const uint8_t* masks, const float* h0, const float* c0, const float* u,
                int32_t* action, float* logp, cudaStream_t s, bool infer) {
  const int N = T * E, Hd = n.H;
  if (N > n.NS || E > n.E) {
    set_error("forward: segment larger than the workspace");
    return DDPPO_E_CONFIG;
  }
  n.enc_valid = false;
  n.lstm_valid = false;
  if (n.F > 0) {
    const int nch = (N + n.NC - 1) / n.NC;
    for (int c = 0; c < nch; ++c) {
      const int r0 = c * n.NC, rn = std::min(n.NC, N - r0);
      DDPPO_TRY(encoder_fwd(n, opoff(n, obs, (size_t)r0 * n.pix), rn,
                            opoff(n, n.featop, (size_t)r0 * n.F), s, infer && n.f8 && rn <= n.E));
    }
    n.ev_valid_chunk = nch - 1;
    GemmDesc v;
    v.M = N; v.N = Hd; v.K = n.F;
    v.A = n.featop; v.lda = n.F; v.B = n.Wv; v.ldb = n.F;
    v.C = n.x1; v.ldc = n.In0; v.c_bf16 = n.bf ? 1 : 0;
    v.bias = n.params + n.vis_b; v.relu = 1;
    DDPPO_TRY(G(n, v, s));
  }
  DDPPO_TRY(launch_embed_fwd(N, goal, prev_a, n.params + n.goal_w, n.params + n.goal_b,
                             n.params + n.emb, n.x1, n.In0, n.emb_col0, n.bf, s));
  DDPPO_TRY(lstm_forward(n, T, E, masks, h0, c0, s));
  Heads hd{};
  hd.N = N; hd.H = Hd; hd.h = n.lstm[n.L - 1].h;
  hd.Wa = n.params + n.actor_w; hd.ba = n.params + n.actor_b;
  hd.Wv = n.params + n.critic_w; hd.bv = n.params + n.critic_b;
  hd.logits = n.logits; hd.value = n.values;
  hd.u = u; hd.action = action; hd.logp = logp;
  DDPPO_TRY(launch_heads_fwd(hd, s));
  n.ev_T = T; n.ev_E = E; n.ev_valid = true;
  n.ev_obs = obs; n.ev_goal = goal; n.ev_preva = prev_a; n.ev_masks = masks;
  n.ev_h0 = h0; n.ev_c0 = c0;
  return DDPPO_OK;
}

int net_backward(Net& n, const float* dlogits, const float* dvalues, cudaStream_t s) {
  if (!n.ev_valid) {
    set_error("policy_backward without a preceding evaluate");
    return DDPPO_E_STATE;
  }
  const int T = n.ev_T, E = n.ev_E, N = T * E, Hd = n.H;
  DDPPO_CHECK_CUDA(cudaMemsetAsync(n.grad, 0, n.P * sizeof(float), s));
  DDPPO_TRY(launch_heads_bwd(N, Hd, n.lstm[n.L - 1].h, n.params + n.actor_w, n.params + n.critic_w,
                             dlogits, dvalues, n.dh_top, n.grad + n.actor_w, n.grad + n.actor_b,
                             n.grad + n.critic_w, n.grad + n.critic_b, n.scratch, n.scratch_elems, s));
  const float* dabove = nullptr;
  DDPPO_TRY(lstm_backward(n, T, E, n.ev_masks, n.ev_c0, n.dh_top, &dabove, s));
  // concatenated LSTM input: [visual FC (H) | goal FC (32) | action embedding (32)]
  DDPPO_TRY(launch_embed_bwd(N, n.ev_goal, n.ev_preva, dabove, n.In0, n.emb_col0,
                             n.grad + n.goal_w, n.grad + n.goal_b, n.grad + n.emb, n.scratch,
                             n.scratch_elems, s));
  if (n.F == 0) return DDPPO_OK;  // blind agent: nothing below the LSTM input
  DDPPO_TRY(launch_vis_relu_bwd(N, Hd, dabove, n.In0, n.x1, n.In0, n.bf, n.dv32, n.dvop, s));
  DDPPO_TRY(launch_colsum(n.dv32, N, Hd, Hd, n.grad + n.vis_b, false, s));
  GemmDesc wv;  // dWv[h, f] = sum_n dv[n, h] feat[n, f]
  wv.M = Hd; wv.N = n.F; wv.K = N;
  wv.A = n.dvop; wv.lda = Hd; wv.a_t = 1; wv.B = n.featop; wv.ldb = n.F; wv.b_t = 1;
  wv.C = n.dWv; wv.ldc = n.F;
  DDPPO_TRY(G(n, wv, s));
  DDPPO_TRY(launch_vis_w_grad(n.dWv, Hd, n.featC, n.featHW, n.grad + n.vis_w, s));
  GemmDesc df;
  df.M = N; df.N = n.F; df.K = Hd;
  df.A = n.dvop; df.lda = Hd; df.B = n.WvT; df.ldb = Hd;
  df.C = n.dfeat; df.ldc = n.F;
  DDPPO_TRY(G(n, df, s));
  DDPPO_TRY(encoder_backward(n, n.ev_obs, N, s));
  return DDPPO_OK;
}


// ---------------------------------------------------------------- stand-alone pieces
// Encoder features leave and enter the library in the parameter layout's order (channel-
// major: f = c * HW + p, the order vis.w's columns use); inside they are NHWC rows.
__global__ void feat_layout_kernel(const float* __restrict__ in, float* __restrict__ out, int N,
                                   int HW, int C, int to_cmajor) {
  DDPPO_PDL_ENTRY();
  const size_t total = (size_t)N * HW * C;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t img = i / ((size_t)HW * C);
    const int r = (int)(i - img * HW * C), p = r / C, c = r - p * C;
    const size_t cm = img * HW * C + (size_t)c * HW + p;
    if (to_cmajor) out[cm] = in[i];
    else out[i] = in[cm];
  }
}

static int feat_layout(const Net& n, const float* in, float* out, int N, bool to_cmajor,
                       cudaStream_t s) {
  const size_t total = (size_t)N * n.F;
  if (!total) return DDPPO_OK;
  const int blocks = (int)std::min<size_t>((total + 255) / 256, 4096);
  ::ddppo::launch_k(feat_layout_kernel, blocks, 256, 0, s, in, out, N, n.featHW, n.featC, to_cmajor ? 1 : 0);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

int net_encoder_forward(Net& n, int N, const void* obs, float* feat, cudaStream_t s) {
  if (n.F == 0) {
    set_error("encoder_forward: the blind agent has no visual encoder");
    return DDPPO_E_CONFIG;
  }
  if (N < 1 || N > n.NS) {
    set_error("encoder_forward: N must be in [1, rollout_T * num_envs / minibatches]");
    return DDPPO_E_CONFIG;
  }
  const int nch = (N + n.NC - 1) / n.NC;
  for (int c = 0; c < nch; ++c) {
    const int r0 = c * n.NC, rn = std::min(n.NC, N - r0);
    DDPPO_TRY(encoder_fwd(n, opoff(n, obs, (size_t)r0 * n.pix), rn,
                          opoff(n, n.featop, (size_t)r0 * n.F), s));
    // the chunk's fp32 features: the post-ReLU output of the last layer
    const float* out = n.kind == 0 ? n.nat[2].z : n.cmp_n.out;
    DDPPO_TRY(feat_layout(n, out, feat + (size_t)r0 * n.F, rn, true, s));
  }
  n.ev_valid_chunk = nch - 1;
  n.ev_valid = false;
  n.lstm_valid = false;
  n.enc_valid = true;
  n.enc_obs = obs;
  n.enc_N = N;
  return DDPPO_OK;
}

int net_encoder_backward(Net& n, const float* dfeat, cudaStream_t s) {
  if (!n.enc_valid) {
    set_error("encoder_backward without a preceding encoder_forward");
    return DDPPO_E_STATE;
  }
  DDPPO_CHECK_CUDA(cudaMemsetAsync(n.grad, 0, n.P * sizeof(float), s));
  DDPPO_TRY(feat_layout(n, dfeat, n.dfeat, n.enc_N, false, s));
  return encoder_backward(n, n.enc_obs, n.enc_N, s);
}

int net_lstm_forward(Net& n, int T, int E, const float* x, const uint8_t* masks, const float* h0,
                     const float* c0, float* y, cudaStream_t s) {
  const int N = T * E;
  if (T < 1 || E < 1 || N > n.NS || E > n.E) {
    set_error("lstm_forward: segment larger than the workspace");
    return DDPPO_E_CONFIG;
  }
  DDPPO_TRY(launch_cast(x, n.x1, n.bf, (size_t)N * n.In0, s));
  DDPPO_TRY(lstm_forward(n, T, E, masks, h0, c0, s));
  DDPPO_CHECK_CUDA(cudaMemcpyAsync(y, n.lstm[n.L - 1].h, (size_t)N * n.H * sizeof(float),
                                   cudaMemcpyDeviceToDevice, s));
  n.ev_valid = false;
  n.enc_valid = false;
  n.lstm_valid = true;
  n.ls_T = T; n.ls_E = E; n.ls_masks = masks; n.ls_c0 = c0;
  return DDPPO_OK;
}

int net_lstm_backward(Net& n, const float* dy, float* dx, cudaStream_t s) {
  if (!n.lstm_valid) {
    set_error("lstm_backward without a preceding lstm_forward");
    return DDPPO_E_STATE;
  }
  const int N = n.ls_T * n.ls_E;
  DDPPO_CHECK_CUDA(cudaMemsetAsync(n.grad, 0, n.P * sizeof(float), s));
  const float* dx0 = nullptr;
  DDPPO_TRY(lstm_backward(n, n.ls_T, n.ls_E, n.ls_masks, n.ls_c0, dy, &dx0, s));
  if (dx)
    DDPPO_CHECK_CUDA(cudaMemcpyAsync(dx, dx0, (size_t)N * n.In0 * sizeof(float),
                                     cudaMemcpyDeviceToDevice, s));
  return DDPPO_OK;
}

}  // namespace ddppo
