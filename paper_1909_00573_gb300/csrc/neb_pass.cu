// neb_pass.cu -- the wavefront kernels of one NEB iteration and their
// orchestration (Sec. 3 outline: pass 1 view paths, pass 2 density / NEE /
// photons, pass 3 self emission).
//
// MIS (Sec. 4): the balance heuristic over the random hit (e), the NEE (E)
// and the NEB photon merges P_k (Eq. rhpdf, Eq. neepdf, Eq. photonpdf,
// Eq. misw) is evaluated recursively.  With F_i = p_{i-1->i}, R_i = p_{i+1->i}
// and ok(k) = [x_k non-delta]:
//   C_m   = sum_{k<m} ok(k) prod_{i=k}^{m-1} R_i / F_{i+1}        (view side)
//   random hit at x_l: p_sum/p_e = 1 + [E] nd(x_{l-1}) q + [P] q rho_{l-1} pi r^2 C_{l-1}, q = p_l / F_l
//   NEE at x_m:        p_sum/p_E = 1 + [e] F_l / p_l + [P] rho_m pi r^2 C_m
//   merge at x_k with a photon from NEE vertex x_m:
//                      p_sum/(n_P p_Pk) = 1 + E0 A_k + B_k + C_k, where the photon
//   carries E0 = ([e] F_l/p_l + [E] nd(x_m)) / (rho_m pi r^2), A_k = prod F_{i+1}/R_i
//   and B_k = sum over photon vertices of ok(k') prod F_{i+1}/R_i.
// n_T cancels (n_P = n_T).  Squared distances cancel between F and R, so only
// cosines and directional pdfs are carried.
#include <cuda_fp16.h>

#include <cfloat>
#include <cstdio>

#include "neb_accum.cuh"
#include "neb_device.cuh"
#include "neb_internal.h"
#include "neb_octree.cuh"

namespace neb {

constexpr int kThreads = 256;

// ---- photon flag word (PhotonRay.mis.w, 16 bits): k of the NEE vertex the
// photon left (0 for light photons), index j of its next hit, light photon,
// light photon before its first hit
constexpr int PH_J_SHIFT = 8, PH_J_MASK = 63;
constexpr int PH_LP = 1 << 14, PH_FIRST = 1 << 15;
constexpr uint32_t kLpStream = 0x40000000u;  // Philox stream of light photon i: + hit index
// Merge mode 0: a photon hit with more view vertices than this in the grid
// cells around it is staged for the per-cell merge; sparser hits merge at once.
constexpr int kStageCandidates = 16;

// ---- photon queue records: PhotonRay (64 bytes) or PackedPhoton (48 bytes)
union Half2Bits {
  __half2 h;
  uint32_t u;
};

__device__ __forceinline__ void store_photon(void* q, int slot, const PhotonRay& ph, int packed) {
  if (!packed) {
    reinterpret_cast<PhotonRay*>(q)[slot] = ph;
    return;
  }
  PackedPhoton pk;
  pk.o = ph.o;
  pk.mis = make_float4(ph.mis.x, ph.mis.y, ph.mis.z, ph.d.w);
  float m = fmaxf(fmaxf(ph.phi.x, ph.phi.y), ph.phi.z);
  int e = 0;
  if (m > 0.0f) frexpf(m, &e);  // m = f 2^e with f in [0.5, 1)
  e = min(max(e, -126), 127);
  const float sc = ldexpf(1.0f, -e);
  Half2Bits rg, bc;
  rg.h = __floats2half2_rn(ph.phi.x * sc, ph.phi.y * sc);
  bc.h = __floats2half2_rn(ph.phi.z * sc, ph.phi.w);
  pk.q = make_uint4(oct_encode16(xyz(ph.d)), rg.u, bc.u,
                    ((uint32_t)__float_as_int(ph.mis.w) & 0xffffu) | ((uint32_t)(e + 128) << 16));
  reinterpret_cast<PackedPhoton*>(q)[slot] = pk;
}

__device__ __forceinline__ PhotonRay load_photon(const void* q, int i, int packed) {
  if (!packed) return reinterpret_cast<const PhotonRay*>(q)[i];
  const PackedPhoton pk = reinterpret_cast<const PackedPhoton*>(q)[i];
  PhotonRay ph;
  float3 d = oct_decode16(pk.q.x);
  const float sc = ldexpf(1.0f, (int)(pk.q.w >> 16) - 128);
  Half2Bits rg, bc;
  rg.u = pk.q.y;
  bc.u = pk.q.z;
  float2 frg = __half22float2(rg.h), fbc = __half22float2(bc.h);
  ph.o = pk.o;
  ph.d = make_float4(d.x, d.y, d.z, pk.mis.w);
  ph.phi = make_float4(frg.x * sc, frg.y * sc, fbc.x * sc, fbc.y);
  ph.mis = make_float4(pk.mis.x, pk.mis.y, pk.mis.z, __int_as_float((int)(pk.q.w & 0xffffu)));
  return ph;
}

// Grid of the shading kernels: SMs x the context's blocks per SM.
static int grid_blocks(const neb_ctx* c) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  return sms * c->tune.shade_blocks_per_sm;
}

// NEE area pdf p_l of point y on light li seen from x (power-proportional
// selection times uniform area on triangles / on the hemisphere of a sphere
// that faces x).
__device__ __forceinline__ float light_pdf(const SceneView& s, int li, float3 y, float3 x) {
  int prim = __ldg(s.light_prim + li);
  float psel = __ldg(s.light_psel + li), ia = __ldg(s.light_inv_area + li);
  if (prim < s.nt) return psel * ia;
  float3 c = xyz(__ldg(s.sph + (prim - s.nt)));
  if (!(dot(sub(y, c), sub(x, c)) > 0.0f)) return 0.0f;
  return psel * ia;
}

// Area pdf of a light point under conventional light-photon emission (Sec.
// 6.1): the light chosen as for NEE, the point uniform on its whole surface
// (a sphere's NEE samples cover the facing hemisphere only: half the pdf).
__device__ __forceinline__ float lp_light_pdf(const SceneView& s, int li) {
  int prim = __ldg(s.light_prim + li);
  float pa = __ldg(s.light_psel + li) * __ldg(s.light_inv_area + li);
  return prim < s.nt ? pa : 0.5f * pa;
}

// Outward (emitting) normal of light li at its point y.
__device__ __forceinline__ float3 light_normal(const SceneView& s, int li, float3 y) {
  int prim = __ldg(s.light_prim + li);
  if (prim < s.nt) {
    float3 v0 = xyz(__ldg(s.tv0 + prim)), v1 = xyz(__ldg(s.tv1 + prim)), v2 = xyz(__ldg(s.tv2 + prim));
    return normalize(cross(sub(v1, v0), sub(v2, v0)));
  }
  return normalize(sub(y, xyz(__ldg(s.sph + (prim - s.nt)))));
}

// ---------------------------------------------------------------------------
// pass 1
// ---------------------------------------------------------------------------
__global__ void k_begin(DevCounters* cnt) {
  cnt->cam_count[1] = 0;
  cnt->nee_count = 0;
  cnt->rh_count = 0;
  cnt->ph_count[0] = 0;
  cnt->ph_count[1] = 0;
  cnt->merge_count = 0;
  cnt->lit_count = 0;
  cnt->shadow_count_b = 0;
  cnt->mh_count = 0;
  cnt->mh_tiles = 0;
  cnt->mh_small = 0;
  cnt->mh_next = 0;
  cnt->mh_next_small = 0;
  cnt->oct_deferred = 0;
}

__global__ void k_camera(IterParams ip, CameraParams cam, CamRay* q, DevCounters* cnt) {
  int P = ip.W * ip.H;
  const bool tiled = (ip.W & 7) == 0 && (ip.H & 3) == 0;
  const int tiles_x = ip.W >> 3;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < P; j += gridDim.x * blockDim.x) {
    // queue order: 8 x 4 pixel tiles, one per warp, when the image is made of them
    const int t = j >> 5, w = j & 31;
    const int pixel = tiled ? ((t / tiles_x) * 4 + (w >> 3)) * ip.W + (t % tiles_x) * 8 + (w & 7) : j;
    uint4 rb = rng_block(ip.key, ip.iteration, pixel, 0, 0);
    float ju = u01(rb.x), jv = u01(rb.y);
    int px = pixel % ip.W, py = pixel / ip.W;
    float sx = (((float)px + ju) / (float)ip.W) * 2.0f - 1.0f;
    float sy = 1.0f - (((float)py + jv) / (float)ip.H) * 2.0f;
    float a = sx * cam.tanh_ * cam.aspect;
    float b = sy * cam.tanh_;
    float3 d = normalize(f3(cam.fwd.x + cam.right.x * a + cam.up.x * b, cam.fwd.y + cam.right.y * a + cam.up.y * b,
                            cam.fwd.z + cam.right.z * a + cam.up.z * b));
    CamRay r;
    r.o = make_float4(cam.eye.x, cam.eye.y, cam.eye.z, __int_as_float(pixel));
    r.d = make_float4(d.x, d.y, d.z, 1.0f);
    r.tau = make_float4(1.0f, 1.0f, 1.0f, 0.0f);
    r.mis = make_float4(0.0f, 0.0f, __int_as_float(-1), __int_as_float(RAY_FROM_CAMERA));
    q[j] = r;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    cnt->cam_count[0] = P;
    atomicAdd(&cnt->camera_rays, 0ull);
  }
}

// Camera path extension: closest hit, random-hit event, NEE vertex (light
// sample, octree-bound record), BSDF sample and the next ray.  Queues are
// compacted with warp ballots.
__global__ void __launch_bounds__(kThreads) k_extend(SceneView s, IterParams ip, int k, const CamRay* __restrict__ in,
                                                     int in_slot, CamRay* __restrict__ out, int out_slot,
                                                     NeeStore nv, RHEvent* __restrict__ rh, DevCounters* cnt,
                                                     int* __restrict__ slot_map, const int2* __restrict__ hits,
                                                     const NeeLight* __restrict__ lights,
                                                     const int2* __restrict__ alias) {
  const int count = min(cnt->cam_count[in_slot], ip.cap_cam);
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x; base < count; base += stride) {
    const int i = base + threadIdx.x;
    const bool valid = i < count;
    uint32_t rays = 0, nee_new = 0, rhits = 0;
    bool store_nee = false, alive = false;
    CamRay ry;
    float3 p = f3(0, 0, 0), n = f3(0, 0, 0), err = f3(0, 0, 0), d = f3(0, 0, 0), tau = f3(0, 0, 0);
    Mat m;
    m.type = 0;
    int pixel = 0, mat = 0, flags = 0;
    float Cfac = 0.0f, cos_k = 0.0f;
    // NEE sample
    float3 ldir = f3(0, 0, 0), dE = f3(0, 0, 0);
    float ldist = 0.0f, g_y = 0.0f;
    bool shadow = false;
    float nee_p_lp = 0.0f;
    int hit_prim = -1;
    // NEE light choice (its alias slot, then the chosen light's record): it
    // depends only on the pixel and k, so these loads go out first and
    // overlap those of the hit
    const bool want_nee = k <= ip.D - 1 && s.nl > 0;
    int lidx = 0, lprim = 0;
    float u2 = 0.0f, u3 = 0.0f, l_pa = 0.0f;
    float4 la0 = make_float4(0, 0, 0, 0), la1 = la0, la2 = la0;  // light triangle, or la0: light sphere
    float3 l_emit = f3(0, 0, 0);
    if (valid) {
      ry = in[i];
      rays = 1;
      d = xyz(ry.d);
      pixel = __float_as_int(ry.o.w);
      flags = __float_as_int(ry.mis.w);
      if (want_nee) {
        uint4 rb = rng_block(ip.key, ip.iteration, pixel, 256u * k, 0);
        lidx = (int)(((uint64_t)(rb.x >> 8) * (uint64_t)s.nl) >> 24);
        const int2 slot = __ldg(alias + lidx);
        if (!(u01(rb.y) < __int_as_float(slot.x))) lidx = slot.y;
        u2 = u01(rb.z);
        u3 = u01(rb.w);
        const NeeLight* L = lights + lidx;
        la0 = __ldg(&L->a);
        la1 = __ldg(&L->b);
        la2 = __ldg(&L->c);
        l_emit = xyz(__ldg(&L->e));
        lprim = __float_as_int(la2.w);
        l_pa = la1.w;
      }
      RayPre r = make_ray(xyz(ry.o), d);
      int2 hh = hits[i];
      int prim = hh.x;
      hit_prim = prim;
      float t = __int_as_float(hh.y);
      if (prim >= 0) {
        hit_point(s, r, prim, t, p, err, n);
        mat = prim_mat(s, prim);
        m = load_mat(s.mats, mat);
        float3 wo = neg(d);
        tau = xyz(ry.tau);
        cos_k = fabsf(dot(n, d));
        int li = __ldg(s.prim_light + prim);
        if ((ip.mask & 1u) && li >= 0 && (prim >= s.nt || dot(n, wo) > 0.0f)) {
          float F_l = (flags & RAY_FROM_CAMERA) ? 0.0f : ry.d.w * cos_k / (t * t);
          int slot = atomicAdd(&cnt->rh_count, 1);
          if (slot < ip.cap_rh) {
            RHEvent e;
            float3 L = cmul(tau, m.emission);
            e.L = make_float4(L.x, L.y, L.z, F_l);
            e.y = make_float4(p.x, p.y, p.z, __int_as_float(li));
            e.info = make_int4(pixel, __float_as_int(ry.mis.z), flags, __float_as_int(ry.mis.y));
            rh[slot] = e;
          } else {
            atomicOr(&cnt->status, NEB_STATUS_QUEUE_OVERFLOW);
          }
          rhits = 1;
        }
        if (!mat_black(m)) {
          alive = k < ip.D;
          Cfac = (flags & RAY_FROM_CAMERA) ? 0.0f : ry.mis.x * ry.tau.w / (ry.d.w * cos_k);
          if (want_nee) {
            store_nee = true;
            nee_new = 1;
            float3 y, ny;
            float p_l;
            if (lprim < s.nt) {
              float b1 = u2, b2 = u3;
              if (b1 + b2 > 1.0f) { b1 = 1.0f - b1; b2 = 1.0f - b2; }
              float3 a0 = xyz(la0), a1 = xyz(la1), a2 = xyz(la2);
              float3 e1 = sub(a1, a0), e2 = sub(a2, a0);
              y = add(add(a0, mul(e1, b1)), mul(e2, b2));
              ny = normalize(cross(e1, e2));
              p_l = l_pa;
            } else {
              float3 ce = xyz(la0);
              float3 w = normalize(sub(p, ce));
              float z = u2;
              float rr = sqrtf(fmaxf(0.0f, 1.0f - z * z));
              float phi = kTwoPi * u3;
              float3 dir = from_local(w, rr * cosf(phi), rr * sinf(phi), z);
              y = add(ce, mul(dir, la0.w));
              ny = dir;
              // the sampled hemisphere faces x: the pdf of light_pdf
              p_l = dot(sub(y, ce), sub(p, ce)) > 0.0f ? l_pa : 0.0f;
            }
            float3 dd = sub(y, p);
            float dist2 = dot(dd, dd);
            float dist = sqrtf(dist2);
            ldir = mul(dd, 1.0f / dist);
            ldist = dist;
            float cos_y = -dot(ny, ldir);
            if (cos_y > 0.0f && p_l > 0.0f) {
              float cos_x = fabsf(dot(n, ldir));
              float g = cos_x * cos_y / (dist2 * p_l);
              dE = mul(l_emit, g);
              g_y = cos_y / (dist2 * p_l);
              shadow = true;
              nee_p_lp = lprim < s.nt ? l_pa : 0.5f * l_pa;  // the light-photon pdf of lp_light_pdf
            }
          }
        }
      }
    }
    // NEE vertex slot (all lanes)
    int nid = warp_append(&cnt->nee_count, store_nee, ip.cap_nee, &cnt->status);
    bool emit = false;
    CamRay nr;
    if (valid && store_nee && nid >= 0) {
      bool delta = mat_delta(m);
      // mergeable: NEB photons reach x_k for k <= D - 2, light photons for k <= D - 1
      const int kmerge = ip.n_lp > 0 ? ip.D - 1 : ip.D - 2;
      int vflags = (delta ? NV_DELTA : 0) | ((!delta && k <= kmerge) ? NV_MERGEABLE : 0) | (shadow ? NV_SHADOW : 0);
      nv.pos[nid] = make_float4(p.x, p.y, p.z, Cfac);
      nv.prim[nid] = hit_prim;
      nv.nrm[nid] = make_float4(n.x, n.y, n.z, __int_as_float(mat | (k << NV_K_SHIFT) | (vflags << NV_FLAG_SHIFT)));
      nv.wo[nid] = make_float4(-d.x, -d.y, -d.z, __int_as_float(pixel));
      nv.tau[nid] = make_float4(tau.x, tau.y, tau.z, g_y);
      nv.err[nid] = make_float4(err.x, err.y, err.z, ldist);
      nv.ldir[nid] = make_float4(ldir.x, ldir.y, ldir.z, -2.0f);  // rho: not evaluated (yet)
      nv.dE[nid] = make_float4(dE.x, dE.y, dE.z, nee_p_lp);
      if (slot_map) slot_map[(size_t)pixel * (ip.D - 1) + (k - 1)] = nid;
    }
    if (valid && alive) {
      float3 wo = neg(d);
      uint4 rb = rng_block(ip.key, ip.iteration, pixel, 256u * k, 1);
      float3 wi, w;
      float pdf_f, pdf_r;
      if (bsdf_sample(m, n, wo, u01(rb.x), u01(rb.y), u01(rb.z), true, wi, w, pdf_f, pdf_r)) {
        float3 nt = cmul(tau, w);
        if (maxc(nt) > 0.0f) {
          float C_k = pdf_r * Cfac;
          bool delta = mat_delta(m);
          float3 o = offset_origin(p, n, err, wi);
          nr.o = make_float4(o.x, o.y, o.z, __int_as_float(pixel));
          nr.d = make_float4(wi.x, wi.y, wi.z, pdf_f);
          nr.tau = make_float4(nt.x, nt.y, nt.z, fabsf(dot(n, wi)));
          nr.mis = make_float4(C_k + (delta ? 0.0f : 1.0f), C_k, __int_as_float(store_nee ? nid : -1),
                               __int_as_float(delta ? RAY_PREV_DELTA : 0));
          emit = true;
        }
      }
    }
    int slot = warp_append(&cnt->cam_count[out_slot], emit, ip.cap_cam, &cnt->status);
    if (emit && slot >= 0) out[slot] = nr;
    warp_count(&cnt->camera_rays, rays);
    warp_count(&cnt->nee_vertices, nee_new);
    warp_count(&cnt->random_hits, rhits);
  }
}

// ---------------------------------------------------------------------------
// pass 2: NEE contributions and photon emission from the NEE vertices
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_nee(SceneView s, IterParams ip, NeeStore nv, DevCounters* cnt,
                                                  double* accum, double* split, void* __restrict__ phq, int packed) {
  // both the NEE contribution and the photon need dE != 0: the kernel walks
  // the list of vertices whose shadow ray reached the light
  const int count = min(cnt->lit_count, ip.cap_nee);
  const int stride = gridDim.x * blockDim.x;
  const int P = ip.W * ip.H;
  const float pir2 = kPi * ip.r * ip.r;
  for (int base = blockIdx.x * blockDim.x; base < count; base += stride) {
    const int t = base + threadIdx.x;
    const int i = t < count ? nv.lit[t] : 0;
    bool emit = false;
    PhotonRay ph;
    uint32_t nphot = 0;
    const float4 de = t < count ? nv.dE[i] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (t < count && maxc(xyz(de)) > 0.0f) {
      float4 pp = nv.pos[i], nn = nv.nrm[i], ww = nv.wo[i], tt = nv.tau[i], ee = nv.err[i], ld = nv.ldir[i];
      int bits = __float_as_int(nn.w);
      int mat = bits & NV_MAT_MASK, k = (bits >> NV_K_SHIFT) & 63, vflags = (bits >> NV_FLAG_SHIFT) & 7;
      bool delta = vflags & NV_DELTA;
      int pixel = __float_as_int(ww.w);
      float3 p = xyz(pp), n = xyz(nn), wo = xyz(ww), tau = xyz(tt), ldir = xyz(ld), dE = xyz(de);
      float rho = ld.w, Cfac = pp.w, g_y = tt.w;
      Mat m = load_mat(s.mats, mat);
      if ((ip.mask & 2u) && !delta) {
        float3 f = bsdf_eval(m, n, wo, ldir);
        if (maxc(f) > 0.0f) {
          float pdfF = bsdf_pdf(m, n, wo, ldir), pdfC = bsdf_pdf(m, n, ldir, wo);
          float inv_w = 1.0f + ((ip.mask & 1u) ? pdfF * g_y : 0.0f) + ((ip.mask & 4u) ? rho * pir2 * pdfC * Cfac : 0.0f);
          // light photons: n_LP pi r^2 p_l^LP R_{l-1} / p_l (C_m + 1), R_{l-1} / p_l = g_y |cos_m| / pi
          if (ip.n_lp > 0)
            inv_w += (float)ip.n_lp * pir2 * de.w * g_y * fabsf(dot(n, ldir)) * kInvPi * (pdfC * Cfac + 1.0f);
          float3 L = mul(cmul(cmul(tau, f), dE), 1.0f / inv_w);
          add_pixel(accum, split, 1, pixel, L, P);
        }
      }
      if ((ip.mask & 4u) && ip.D >= 3 && rho > 0.0f) {
        float3 phi0 = mul(dE, 1.0f / rho);
        uint4 rb = rng_block(ip.key, ip.iteration, pixel, 256u * k + 1u, 1);
        float3 w1, wt;
        float pdf1, pdfr1;
        if (bsdf_sample(m, n, ldir, u01(rb.x), u01(rb.y), u01(rb.z), false, w1, wt, pdf1, pdfr1)) {
          float3 phi = cmul(phi0, wt);
          if (maxc(phi) > 0.0f) {
            float E0 = (((ip.mask & 1u) ? pdfr1 * g_y : 0.0f) + (((ip.mask & 2u) && !delta) ? 1.0f : 0.0f)) /
                       (rho * pir2);
            if (ip.n_lp > 0) {
              // alpha / (rho pi r^2) = 1 + lp and beta gains lp ok(x_m), lp = n_LP p_l^LP
              // R_{l-1} / (p_l rho); both are divided out: flux / alpha, E0 = beta / alpha
              float lp = (float)ip.n_lp * de.w * g_y * fabsf(dot(n, ldir)) * kInvPi / rho;
              float a = 1.0f + lp;
              E0 = (E0 + (delta ? 0.0f : lp)) / a;
              phi = mul(phi, 1.0f / a);
            }
            float3 o = offset_origin(p, n, xyz(ee), w1);
            ph.o = make_float4(o.x, o.y, o.z, __int_as_float(pixel));
            ph.d = make_float4(w1.x, w1.y, w1.z, pdf1);
            ph.phi = make_float4(phi.x, phi.y, phi.z, fabsf(dot(n, w1)));
            ph.mis = make_float4(E0, 1.0f, 0.0f, __int_as_float(k | (1 << 8)));
            emit = true;
            nphot = 1;
          }
        }
      }
    }
    int slot = warp_append(&cnt->ph_count[0], emit, ip.cap_ph, &cnt->status);
    if (emit && slot >= 0) store_photon(phq, slot, ph, packed);
    warp_count(&cnt->photons, nphot);
  }
}

// Conventional light photons (Sec. 6.1): n_LP photons per iteration, each
// from a light chosen as for NEE (alias table, Philox dims 0-1 of stream
// kLpStream), a point uniform on its whole surface (dims 2-3) and a direction
// cosine-weighted about its normal (dims 4-5), with flux Le cos / (p_l^LP
// cos / pi) / n_LP.  They follow the NEB photons in the photon queue; their
// weights are set up at their first hit (k_photon).
__global__ void __launch_bounds__(kThreads) k_lp_emit(SceneView s, IterParams ip, DevCounters* cnt,
                                                      void* __restrict__ phq, int packed) {
  for (int base = blockIdx.x * blockDim.x; base < ip.n_lp; base += gridDim.x * blockDim.x) {
    const int i = base + threadIdx.x;
    bool emit = false;
    PhotonRay ph;
    if (i < ip.n_lp && s.nl > 0) {
      uint4 r0 = rng_block(ip.key, ip.iteration, i, kLpStream, 0);
      uint4 r1 = rng_block(ip.key, ip.iteration, i, kLpStream, 1);
      int li = (int)(((uint64_t)(r0.x >> 8) * (uint64_t)s.nl) >> 24);
      if (!(u01(r0.y) < __ldg(s.alias_prob + li))) li = __ldg(s.alias_idx + li);
      const int prim = __ldg(s.light_prim + li);
      const float u2 = u01(r0.z), u3 = u01(r0.w);
      float3 y, ny, yerr;
      if (prim < s.nt) {
        float b1 = u2, b2 = u3;
        if (b1 + b2 > 1.0f) { b1 = 1.0f - b1; b2 = 1.0f - b2; }
        float3 a = xyz(__ldg(s.tv0 + prim)), e1 = sub(xyz(__ldg(s.tv1 + prim)), a), e2 = sub(xyz(__ldg(s.tv2 + prim)), a);
        y = add(add(a, mul(e1, b1)), mul(e2, b2));
        ny = normalize(cross(e1, e2));
        yerr = f3(NEB_GAMMA5 * (fabsf(a.x) + fabsf(e1.x * b1) + fabsf(e2.x * b2)),
                  NEB_GAMMA5 * (fabsf(a.y) + fabsf(e1.y * b1) + fabsf(e2.y * b2)),
                  NEB_GAMMA5 * (fabsf(a.z) + fabsf(e1.z * b1) + fabsf(e2.z * b2)));
      } else {
        float4 sp = __ldg(s.sph + (prim - s.nt));
        float z = 1.0f - 2.0f * u2;
        float rr = sqrtf(fmaxf(0.0f, 1.0f - z * z));
        float phs = kTwoPi * u3;
        ny = f3(rr * cosf(phs), rr * sinf(phs), z);
        y = add(xyz(sp), mul(ny, sp.w));
        yerr = f3(NEB_GAMMA5 * (fabsf(sp.x) + sp.w), NEB_GAMMA5 * (fabsf(sp.y) + sp.w),
                  NEB_GAMMA5 * (fabsf(sp.z) + sp.w));
      }
      const float u4 = u01(r1.x), u5 = u01(r1.y);
      const float er = sqrtf(u4), eph = kTwoPi * u5, ez = sqrtf(fmaxf(0.0f, 1.0f - u4));
      float3 w = from_local(ny, er * cosf(eph), er * sinf(eph), ez);
      if (ez > 0.0f) {
        const float p_lp = lp_light_pdf(s, li);
        Mat lm = load_mat(s.mats, prim_mat(s, prim));
        float3 phi = mul(lm.emission, kPi / (p_lp * (float)ip.n_lp));
        float3 o = offset_origin(y, ny, yerr, w);
        ph.o = make_float4(o.x, o.y, o.z, __int_as_float(i));
        ph.d = make_float4(w.x, w.y, w.z, 1.0f);
        ph.phi = make_float4(phi.x, phi.y, phi.z, ez);  // w: cos_y
        ph.mis = make_float4(p_lp, __int_as_float(li), 0.0f, __int_as_float((1 << PH_J_SHIFT) | PH_LP | PH_FIRST));
        emit = true;
      }
    }
    int slot = warp_append(&cnt->ph_count[0], emit, ip.cap_ph, &cnt->status);
    if (emit && slot >= 0) store_photon(phq, slot, ph, packed);
    warp_count(&cnt->photons, emit ? 1u : 0u);
  }
}

// pass 3: self emission of the stored random hits (Sec. 3.3)
__global__ void __launch_bounds__(kThreads) k_emission(SceneView s, IterParams ip, NeeStore nv, const RHEvent* rh,
                                                       DevCounters* cnt, double* accum, double* split,
                                                       const int* __restrict__ oct_nodes, const OctreeState* oct_state,
                                                       OctreeParams oct, int robust) {
  const int count = min(cnt->rh_count, ip.cap_rh);
  const int P = ip.W * ip.H;
  const float pir2 = kPi * ip.r * ip.r;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
    RHEvent ev = rh[e];
    int pixel = ev.info.x, prev = ev.info.y, flags = ev.info.z;
    float C_prev = __int_as_float(ev.info.w);
    float inv_w = 1.0f;
    if (!(flags & RAY_FROM_CAMERA)) {
      float rho = 0.0f;
      float3 xp;
      if (prev >= 0) {
        const float4 xp4 = nv.pos[prev];
        xp = xyz(xp4);
        rho = nv.ldir[prev].w;
        if (rho < -1.5f) {  // not evaluated by the density pass (its shadow ray was blocked)
          const float4 nn = nv.nrm[prev];
          const float pp[3] = {xp4.x, xp4.y, xp4.z}, qq[3] = {nn.x, nn.y, nn.z};
          int queries = 0;
          rho = robust ? oct_density_robust(oct_nodes, oct, pp, qq, &queries) : oct_density(oct_nodes, oct, pp, qq);
        }
      } else {
        continue;  // the NEE store overflowed; the event cannot be weighted
      }
      const int li = __float_as_int(ev.y.w);
      float p_l = light_pdf(s, li, xyz(ev.y), xp);
      float q = p_l / ev.L.w;
      inv_w = 1.0f + (((ip.mask & 2u) && !(flags & RAY_PREV_DELTA)) ? q : 0.0f) +
              ((ip.mask & 4u) ? q * rho * pir2 * C_prev : 0.0f);
      if (ip.n_lp > 0) {
        // light photons: n_LP pi r^2 p_l^LP R_{l-1} / F_l (C_{l-1} + ok(x_{l-1})), with
        // R_{l-1} = (cos_y / pi) |cos_{l-1}| / d^2 the cosine emission toward x_{l-1}
        float3 y = xyz(ev.y), dd = sub(y, xp);
        float d2 = dot(dd, dd);
        float3 u = mul(dd, rsqrtf(d2));
        float cos_y = -dot(light_normal(s, li, y), u);
        float cos_p = fabsf(dot(xyz(nv.nrm[prev]), u));
        if (cos_y > 0.0f) {
          float R = cos_y * kInvPi * cos_p / d2;
          inv_w += (float)ip.n_lp * pir2 * lp_light_pdf(s, li) * R / ev.L.w *
                   (C_prev + ((flags & RAY_PREV_DELTA) ? 0.0f : 1.0f));
        }
      }
    }
    float3 L = mul(xyz(ev.L), 1.0f / inv_w);
    add_pixel(accum, split, 0, pixel, L, P);
  }
}

// Photon walk: closest hit, merge with the view vertices of the hashed grid
// (inverted search of Sec. 3.2), then the next scattering.
__global__ void __launch_bounds__(kThreads) k_photon(SceneView s, IterParams ip, int j, const void* __restrict__ in,
                                                     int in_slot, void* __restrict__ out, int out_slot, int packed,
                                                     NeeStore nv, const MergeRec* __restrict__ mrec,
                                                     const int* __restrict__ bucket_start, DevCounters* cnt,
                                                     double* accum, double* split, const int2* __restrict__ hits,
                                                     const int* __restrict__ oct_nodes, const OctreeState* oct_state,
                                                     OctreeParams oct, int robust, MergeHit* __restrict__ mh) {
  const int count = min(cnt->ph_count[in_slot], ip.cap_ph);
  const int stride = gridDim.x * blockDim.x;
  const int P = ip.W * ip.H;
  for (int base = blockIdx.x * blockDim.x; base < count; base += stride) {
    const int i = base + threadIdx.x;
    bool emit = false;
    PhotonRay nph;
    uint32_t nhits = 0, tests = 0, merges = 0;
    bool want_merge = false;
    float3 m_p = f3(0, 0, 0), m_d = f3(0, 0, 0), m_phi = f3(0, 0, 0);
    // merge weight of this hit: 1 / w = c0 + c1 pdfF + c2 pdfC Cfac, for view
    // vertices x_k with k <= kmax, contributions to split channel chan
    float m_c0 = 0.0f, m_c1 = 0.0f, m_c2 = 0.0f;
    int m_kmax = -1, m_chan = 2;
    int queries = 0;
    if (i < count) {
      PhotonRay ph = load_photon(in, i, packed);
      float3 d = xyz(ph.d);
      RayPre r = make_ray(xyz(ph.o), d);
      int2 hh = hits[i];
      int prim = hh.x;
      float t = __int_as_float(hh.y);
      if (prim >= 0) {
        float3 hp, herr, hn;
        hit_point(s, r, prim, t, hp, herr, hn);
        Mat hm = load_mat(s.mats, prim_mat(s, prim));
        if (!mat_black(hm)) {
          nhits = 1;
          const int bits = __float_as_int(ph.mis.w);
          const int knee = bits & 0xff, jph = (bits >> PH_J_SHIFT) & PH_J_MASK;
          const bool lp = bits & PH_LP;
          int pixel = __float_as_int(ph.o.w);
          float cos_hit = fabsf(dot(hn, d));
          float3 phi = xyz(ph.phi);
          bool hdelta = mat_delta(hm);
          const float pir2 = kPi * ip.r * ip.r;
          if (bits & PH_FIRST) {
            // First hit x_{l-1} of a light photon from the light point y (Sec. 6.1).
            // Every LP path of this photon ends here: with R = p_{l -> l-1} (cosine
            // emission), p_l the NEE pdf of y from here and rho the density here,
            // num = n_LP pi r^2 (p_l^LP / p_l) R is the light-photon strategy,
            // alpha = [P] rho pi r^2 + num the coefficient of the interior merges and
            // beta = [E] + [e] F_l / p_l + num that of this vertex (Q normalisation).
            const float3 yl = xyz(ph.o);
            const float3 dl = sub(hp, yl);
            const float d2 = dot(dl, dl);
            const float cos_y = ph.phi.w, p_lp = ph.mis.x;
            const int li = __float_as_int(ph.mis.y);
            const float p_l = light_pdf(s, li, yl, hp);
            float pp[3] = {hp.x, hp.y, hp.z}, nn[3] = {hn.x, hn.y, hn.z};
            const float rho = robust ? oct_density_robust(oct_nodes, oct, pp, nn, &queries)
                                     : (++queries, oct_density(oct_nodes, oct, pp, nn));
            if (p_l > 0.0f) {
              const float R = cos_y * kInvPi * cos_hit / d2;
              const float num = (float)ip.n_lp * pir2 * (p_lp / p_l) * R;
              const float alpha = ((ip.mask & 4u) ? rho * pir2 : 0.0f) + num;
              const float g = cos_y / (d2 * p_l);  // F_l / p_l = pdfF g
              if (!hdelta) {
                // merging here: x_k stands for x_{l-1}; beta per view vertex
                want_merge = true;
                m_p = hp;
                m_d = d;
                m_phi = phi;
                m_c0 = ((ip.mask & 2u) ? 1.0f / num : 0.0f) + 1.0f;
                m_c1 = (ip.mask & 1u) ? g / num : 0.0f;
                m_c2 = alpha / num;
                m_kmax = ip.D - 1;
                m_chan = 3;
              }
              if (j + 1 <= ip.D - 1) {
                // leave x_{l-1} as a photon emitted there, with 1 / alpha folded
                // into its flux and beta / alpha as its E0
                uint4 rb = rng_block(ip.key, ip.iteration, pixel, kLpStream + (uint32_t)j, 1);
                float3 w, wt;
                float pdf_f, pdf_r;
                if (bsdf_sample(hm, hn, neg(d), u01(rb.x), u01(rb.y), u01(rb.z), false, w, wt, pdf_f, pdf_r)) {
                  float3 phi2 = mul(cmul(phi, wt), num / alpha);
                  if (maxc(phi2) > 0.0f && alpha > 0.0f) {
                    float beta = (((ip.mask & 2u) && !hdelta) ? 1.0f : 0.0f) + ((ip.mask & 1u) ? pdf_r * g : 0.0f) +
                                 (hdelta ? 0.0f : num);
                    float3 o = offset_origin(hp, hn, herr, w);
                    nph.o = make_float4(o.x, o.y, o.z, __int_as_float(pixel));
                    nph.d = make_float4(w.x, w.y, w.z, pdf_f);
                    nph.phi = make_float4(phi2.x, phi2.y, phi2.z, fabsf(dot(hn, w)));
                    nph.mis = make_float4(beta / alpha, 1.0f, 0.0f, __int_as_float((1 << PH_J_SHIFT) | PH_LP));
                    emit = true;
                  }
                }
              }
            }
          } else {
            // NEB photons, and light photons after their first hit
            float cos_orig = ph.phi.w, pdf_dir = ph.d.w;
            float E0 = ph.mis.x, pA = ph.mis.y, pB = ph.mis.z;
            if (!hdelta) {
              want_merge = true;
              m_p = hp;
              m_d = d;
              m_phi = phi;
              m_c0 = 1.0f;
              m_c1 = (E0 * pA + pB) * cos_orig / (pdf_dir * cos_hit);
              m_c2 = 1.0f;
              m_kmax = ip.D - jph - 1;
              m_chan = lp ? 3 : 2;
            }
            if (jph + 1 <= ip.D - 2) {
              const uint32_t stream = lp ? kLpStream + (uint32_t)j : 256u * knee + 1u + (uint32_t)j;
              uint4 rb = rng_block(ip.key, ip.iteration, pixel, stream, 1);
              float3 w, wt;
              float pdf_f, pdf_r;
              if (bsdf_sample(hm, hn, neg(d), u01(rb.x), u01(rb.y), u01(rb.z), false, w, wt, pdf_f, pdf_r)) {
                float3 phi2 = cmul(phi, wt);
                if (maxc(phi2) > 0.0f) {
                  float ratio = pdf_r * cos_orig / (pdf_dir * cos_hit);
                  float3 o = offset_origin(hp, hn, herr, w);
                  nph.o = make_float4(o.x, o.y, o.z, __int_as_float(pixel));
                  nph.d = make_float4(w.x, w.y, w.z, pdf_f);
                  nph.phi = make_float4(phi2.x, phi2.y, phi2.z, fabsf(dot(hn, w)));
                  nph.mis = make_float4(E0, ratio * pA, (hdelta ? 0.0f : 1.0f) + ratio * pB,
                                        __int_as_float(knee | ((jph + 1) << PH_J_SHIFT) | (lp ? PH_LP : 0)));
                  emit = true;
                }
              }
            }
          }
        }
      }
    }
    // Merge (inverted range search, Sec. 3.2).  Each lane looks up the bucket
    // ranges of its own hit's eight cells (all loads in flight at once), a
    // warp scan lays the candidate lists of the 32 hits end to end, and the
    // lanes take that combined list 32 entries at a time: lane l handles entry
    // 32 q + l, whose hit and cell it finds by a binary search over the
    // scanned counts.  A hit in a dense cell is thus spread over the warp and
    // no hit waits for the lookups of another.
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int cb[8], cl[8];  // bucket start and length of each cell (0 for a repeated bucket)
    int nl = 0;
    if (want_merge) {
      float gx = (m_p.x - ip.gmin.x) * ip.cell_inv, gy = (m_p.y - ip.gmin.y) * ip.cell_inv,
            gz = (m_p.z - ip.gmin.z) * ip.cell_inv;
      int cx = grid_cell_index(gx), cy = grid_cell_index(gy), cz = grid_cell_index(gz);
      int ox = (gx - (float)cx >= 0.5f) ? 1 : -1, oy = (gy - (float)cy >= 0.5f) ? 1 : -1,
          oz = (gz - (float)cz >= 0.5f) ? 1 : -1;
      uint32_t bk[8];
      bool occ[8];  // the cell holds a mergeable vertex (its occupancy bit)
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int x = cx + ((c & 1) ? ox : 0), y = cy + ((c & 2) ? oy : 0), z = cz + ((c & 4) ? oz : 0);
        bk[c] = grid_hash(x, y, z, ip.table_mask);
        occ[c] = cell_occupied(ip.cell_bits, ip.cell_bits_mask, x, y, z);
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        bool dup = false;
#pragma unroll
        for (int c2 = 0; c2 < c; ++c2) dup |= occ[c2] && bk[c2] == bk[c];
        int b0 = 0, b1 = 0;
        if (occ[c] && !dup) {
          b0 = __ldg(bucket_start + bk[c]);
          b1 = __ldg(bucket_start + bk[c] + 1);
        }
        cb[c] = b0;
        cl[c] = b1 - b0;
        nl += cl[c];
      }
    } else {
#pragma unroll
      for (int c = 0; c < 8; ++c) cb[c] = cl[c] = 0;
    }
    // A hit with many view vertices in its cells is staged for the per-cell
    // merge that follows the last photon walk (if the list has room); the
    // others merge here.
    if (ip.cap_mh > 0) {
      const bool dense = want_merge && nl > ip.stage_min;
      const unsigned sm = __ballot_sync(0xffffffffu, dense);
      if (sm) {
        const int leader = __ffs(sm) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(&cnt->mh_count, __popc(sm));
        base = __shfl_sync(0xffffffffu, base, leader);
        const int slot = base + __popc(sm & ((1u << lane) - 1u));
        if (dense && slot < ip.cap_mh) {
          MergeHit h;
          h.key = make_float4(m_p.x, m_p.y, m_p.z, __int_as_float((m_kmax & 0xff) | ((m_chan - 2) << 8)));
          h.dir = make_float4(-m_d.x, -m_d.y, -m_d.z, m_c1 / m_c0);
          h.phi = make_float4(m_phi.x / m_c0, m_phi.y / m_c0, m_phi.z / m_c0, m_c2 / m_c0);
          mh[slot] = h;
          nl = 0;
#pragma unroll
          for (int c = 0; c < 8; ++c) cl[c] = 0;
        }
      }
    }
    int incl = nl;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    for (int q0 = 0; q0 < total; q0 += 32) {
      const int q = q0 + lane;
      // owner = number of lanes whose inclusive count is <= q
      int L = 0;
#pragma unroll
      for (int st = 16; st > 0; st >>= 1) {
        int v = __shfl_sync(FULL, incl, L + st - 1);
        if (v <= q) L += st;
      }
      L = L < 31 ? L : 31;
      int u = q - (__shfl_sync(FULL, incl, L) - __shfl_sync(FULL, nl, L));
      int e = -1;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        int len = __shfl_sync(FULL, cl[c], L), start = __shfl_sync(FULL, cb[c], L);
        if (e < 0) {
          if (u < len) e = start + u;
          else u -= len;
        }
      }
      float3 hp = f3(__shfl_sync(FULL, m_p.x, L), __shfl_sync(FULL, m_p.y, L), __shfl_sync(FULL, m_p.z, L));
      float3 md = f3(-__shfl_sync(FULL, m_d.x, L), -__shfl_sync(FULL, m_d.y, L), -__shfl_sync(FULL, m_d.z, L));
      float3 phi = f3(__shfl_sync(FULL, m_phi.x, L), __shfl_sync(FULL, m_phi.y, L), __shfl_sync(FULL, m_phi.z, L));
      float c0 = __shfl_sync(FULL, m_c0, L), c1 = __shfl_sync(FULL, m_c1, L), c2 = __shfl_sync(FULL, m_c2, L);
      int kmax = __shfl_sync(FULL, m_kmax, L), chan = __shfl_sync(FULL, m_chan, L);
      if (q >= total || e < 0) continue;
      float4 mp = __ldg(&mrec[e].pos);
      float dx = mp.x - hp.x, dy = mp.y - hp.y, dz = mp.z - hp.z;
      float d2 = dx * dx + dy * dy + dz * dz;
      ++tests;
      if (!(d2 <= ip.r2)) continue;
      const int id = __float_as_int(mp.w);  // the view vertex, from the NEE store
      float4 mn = __ldg(&nv.nrm[id]);
      int mb = __float_as_int(mn.w);
      int kk = (mb >> NV_K_SHIFT) & 63;
      if (kk > kmax) continue;
      Mat cm = load_mat(s.mats, mb & NV_MAT_MASK);
      float4 mw = __ldg(&nv.wo[id]);
      float3 cn = xyz(mn), cwo = xyz(mw);
      float3 f = bsdf_eval(cm, cn, cwo, md);
      if (!(maxc(f) > 0.0f)) continue;
      float pdfF = bsdf_pdf(cm, cn, cwo, md), pdfC = bsdf_pdf(cm, cn, md, cwo);
      float inv_w = c0 + c1 * pdfF + c2 * pdfC * __ldg(&nv.pos[id].w);
      float3 ctau = xyz(__ldg(&nv.tau[id]));
      float3 L3 = mul(cmul(cmul(ctau, f), phi), ip.kernel / inv_w);
      add_pixel(accum, split, chan, __float_as_int(mw.w), L3, P);
      ++merges;
    }
    int slot = warp_append(&cnt->ph_count[out_slot], emit, ip.cap_ph, &cnt->status);
    if (emit && slot >= 0) store_photon(out, slot, nph, packed);
    warp_count(&cnt->photon_hits, nhits);
    warp_count(&cnt->octree_queries, (uint32_t)queries);
    warp_count(&cnt->merge_tests, tests);
    warp_count(&cnt->merges, merges);
  }
}

__global__ void k_reset_photon_slot(DevCounters* cnt, int slot) { cnt->ph_count[slot] = 0; }
__global__ void k_reset_cam_slot(DevCounters* cnt, int slot) { cnt->cam_count[slot] = 0; }

// image = (sum of the even-iteration half + sum of the odd-iteration half) / iterations
__global__ void k_resolve(const double* __restrict__ accum, int n, double inv, float* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = (float)((accum[i] + accum[n + i]) * inv);
}

// the FP64 sums over all iterations: the two halves added
__global__ void k_sum_halves(const double* __restrict__ accum, int n, double* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = accum[i] + accum[n + i];
}

// Two-half error estimate of the progressive image: with m_e and m_o the
// per-pixel means of the n_e even and n_o odd iterations (luminance, the sum
// of the three channels), the variance of the mean of all n iterations is
// Var(m_e - m_o) n_e n_o / n^2.  The block sums of (m_e - m_o)^2 and of the
// squared mean are added into out[0] and out[1].
__global__ void k_error_sums(const double* __restrict__ accum, int P, int n_even, int n_odd, double* out) {
  __shared__ double s_num[8], s_den[8];
  const double ie = 1.0 / n_even, io = 1.0 / n_odd, in = 1.0 / (n_even + n_odd);
  double num = 0.0, den = 0.0;
  const size_t half = 3 * (size_t)P;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
    const double* e = accum + 3 * (size_t)i;
    const double* o = e + half;
    const double le = e[0] + e[1] + e[2], lo = o[0] + o[1] + o[2];
    const double d = le * ie - lo * io, m = (le + lo) * in;
    num += d * d;
    den += m * m;
  }
  for (int off = 16; off > 0; off >>= 1) {
    num += __shfl_down_sync(0xffffffffu, num, off);
    den += __shfl_down_sync(0xffffffffu, den, off);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_num[w] = num;
    s_den[w] = den;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      a += s_num[k];
      b += s_den[k];
    }
    atomicAdd(out, a);
    atomicAdd(out + 1, b);
  }
}

__global__ void k_fill(float* out, size_t n, float v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) out[i] = v;
}

__global__ void k_read_rho(NeeStore nv, const DevCounters* cnt, int D, int cap_nee, float* out) {
  int count = min(cnt->nee_count, cap_nee);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    int bits = __float_as_int(nv.nrm[i].w);
    int k = (bits >> NV_K_SHIFT) & 63;
    int pixel = __float_as_int(nv.wo[i].w);
    out[(size_t)pixel * (D - 1) + (k - 1)] = nv.ldir[i].w;
  }
}

// ---------------------------------------------------------------------------
// orchestration
// ---------------------------------------------------------------------------
struct StageTimer {
  neb_ctx* c;
  int idx = 0;
  int stage[kMaxStageRecords];
  explicit StageTimer(neb_ctx* ctx) : c(ctx) {}
  void begin(int s) {
    if (!c->profiling || idx >= kMaxStageRecords) return;
    stage[idx] = s;
    cudaEventRecord(c->ev[2 * idx], c->stream);
  }
  void end() {
    if (!c->profiling || idx >= kMaxStageRecords) return;
    cudaEventRecord(c->ev[2 * idx + 1], c->stream);
    ++idx;
  }
  void collect() {
    if (!c->profiling) return;
    cudaEventSynchronize(c->ev[2 * idx - 1]);
    for (int i = 0; i < idx; ++i) {
      float ms = 0;
      cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]);
      c->stage_ms[stage[i]] += ms;
      c->stage_launches[stage[i]] += 1;
    }
  }
};

IterParams iter_params(const neb_ctx* c, int iteration) {
  IterParams ip;
  ip.W = c->W;
  ip.H = c->H;
  ip.D = c->D;
  ip.iteration = iteration;
  ip.key = make_uint2((uint32_t)(c->cfg.seed & 0xffffffffu), (uint32_t)(c->cfg.seed >> 32));
  ip.r = c->cfg.merge_radius;
  ip.r2 = ip.r * ip.r;
  ip.kernel = (float)(1.0 / (3.14159265358979323846 * (double)ip.r * (double)ip.r));
  ip.mask = c->cfg.strategy_mask;
  ip.n_lp = (ip.mask & 8u) ? c->cfg.lp_photons : 0;
  ip.keep_split = c->cfg.keep_split;
  ip.cap_cam = c->cap_cam;
  ip.cap_nee = c->cap_nee;
  ip.cap_rh = c->cap_rh;
  ip.cap_ph = c->cap_ph;
  float cs = 2.0f * ip.r;
  ip.gmin = f3(c->bmin[0] - cs, c->bmin[1] - cs, c->bmin[2] - cs);
  ip.cell_inv = 1.0f / cs;
  ip.table_mask = c->table_size - 1;
  ip.cell_bits = c->cell_bits;
  ip.cell_bits_mask = 32u * c->table_size - 1u;
  ip.cap_mh = c->cap_mh;
  ip.stage_min = c->cfg.merge_mode == 2 ? -1 : kStageCandidates;
  return ip;
}

// Pass 1 of `iteration` on stream st: view paths, NEE samples and shadow rays
// into slot iteration & 1.  Returns the number of kernels enqueued.
static long long enqueue_pass1(neb_ctx* c, int iteration, cudaStream_t st, StageTimer& tm) {
  const int B = grid_blocks(c);
  SceneView s = scene_view(c);
  IterParams ip = iter_params(c, iteration);
  IterSlot& sl = c->slots[iteration & 1];
  DevCounters* cnt = sl.cnt;
  long long launches = 0;
  tm.begin(STAGE_REARM);
  k_begin<<<1, 1, 0, st>>>(cnt);
  if (sl.slot_map) cudaMemsetAsync(sl.slot_map, 0xff, sizeof(int) * (size_t)c->P * (c->D - 1), st);
  launches += 1;
  tm.end();
  tm.begin(STAGE_CAMERA);
  k_camera<<<capped_blocks(c->P, kThreads, B), kThreads, 0, st>>>(ip, c->cam, c->camq[0], cnt);
  launches += 1;
  tm.end();
  for (int k = 1; k <= c->D; ++k) {
    int in = (k - 1) & 1, out = k & 1;
    k_reset_cam_slot<<<1, 1, 0, st>>>(cnt, out);
    // bounce rays are regrouped by origin and direction cell (primary rays
    // are coherent in pixel order already)
    const CamRay* qin = c->camq[in];
    if (k >= 2) {
      tm.begin(STAGE_GROUP);
      launch_group_camera(c, qin, &cnt->cam_count[in], c->camq_grouped, st);
      qin = c->camq_grouped;
      launches += 3;
      tm.end();
    }
    tm.begin(STAGE_TRACE_CAM);
    launch_trace_closest(c, reinterpret_cast<const float4*>(qin), &cnt->cam_count[in], c->cap_cam, c->hits, 0, cnt,
                         st);
    tm.end();
    tm.begin(STAGE_EXTEND);
    k_extend<<<capped_blocks(c->cap_cam, kThreads, B), kThreads, 0, st>>>(
        s, ip, k, qin, in, c->camq[out], out, sl.nv, sl.rh, cnt, sl.slot_map, c->hits, c->nee_lights, c->alias_slots);
    launches += 3;
    tm.end();
  }
  tm.begin(STAGE_GROUP);
  launch_group_shadow(c, sl, st);
  launches += 3;
  tm.end();
  tm.begin(STAGE_SHADOW);
  launch_trace_shadow(c, sl, st);
  launches += shadow_walk_launches(c);
  tm.end();
  return launches;
}

// Passes 2-3 of `iteration` on stream st: the octree's iteration start (Sec.
// 5.4: host-side scalars, device re-arm of the free words), inserts of the iteration's NEE vertices,
// densities, NEE contributions and photon emission; then the deferred random
// hits, photon walks and merges.
static long long enqueue_pass23(neb_ctx* c, int iteration, cudaStream_t st2, StageTimer& tm) {
  const int B = grid_blocks(c);
  SceneView s = scene_view(c);
  IterParams ip = iter_params(c, iteration);
  IterSlot& sl = c->slots[iteration & 1];
  DevCounters* cnt = sl.cnt;
  double* split = c->cfg.keep_split ? c->split : nullptr;
  // iterations of each parity add to their own half of the FP64 sums (the
  // two halves give the error estimate; the image is their sum)
  double* accum = c->accum + (size_t)(iteration & 1) * 3 * (size_t)c->P;
  long long launches = 0;
  octree_set_iteration_params(c->oct, c->cfg.split_factor, iteration);
  tm.begin(STAGE_INSERT);
  if (split) cudaMemsetAsync(c->split, 0, sizeof(double) * 12 * (size_t)c->P, st2);
  launch_oct_rearm(c->oct_nodes, c->oct_state, c->oct, st2);
  launch_oct_insert_nee(c, sl, st2);
  launches += c->cfg.octree_mode == 1 ? 2 : 3;
  tm.end();
  tm.begin(STAGE_DENSITY);
  launch_oct_density_nee(c, sl, st2);
  tm.end();
  tm.begin(STAGE_NEE);
  k_nee<<<capped_blocks(c->cap_nee, kThreads, B), kThreads, 0, st2>>>(s, ip, sl.nv, cnt, accum, split, c->phq[0],
                                                                        c->cfg.photon_records);
  if (ip.n_lp > 0 && c->D >= 2) {
    k_lp_emit<<<capped_blocks(ip.n_lp, kThreads, B), kThreads, 0, st2>>>(s, ip, cnt, c->phq[0], c->cfg.photon_records);
    launches += 1;
  }
  tm.end();
  launches += 2;
  // photon walks: NEB photons hit at most D - 2 times, light photons D - 1 times
  const bool photons = ((ip.mask & 4u) && c->D >= 3) || (ip.n_lp > 0 && c->D >= 2);
  const int photon_launches = ip.n_lp > 0 ? c->D - 1 : c->D - 2;
  if (photons) {
    tm.begin(STAGE_GRID);
    grid_build(c, ip, sl, st2);
    launches += 2 + scan_launch_count((size_t)c->table_size + 1);
    tm.end();
  }
  tm.begin(STAGE_EMISSION);
  k_emission<<<capped_blocks(c->cap_rh, kThreads, B), kThreads, 0, st2>>>(s, ip, sl.nv, sl.rh, cnt, accum, split,
                                                                           c->oct_nodes, c->oct_state, c->oct,
                                                                           c->cfg.density_mode == 0);
  launches += 1;
  tm.end();
  if (photons) {
    for (int j = 1; j <= photon_launches; ++j) {
      int in = (j - 1) & 1, out = j & 1;
      k_reset_photon_slot<<<1, 1, 0, st2>>>(cnt, out);
      const void* qin = c->phq[in];
      if (c->phq_grouped && c->tune.photon_grouping) {
        // photon rays regrouped by origin and direction cell, as the camera
        // bounce rays are, so a warp's rays walk the same nodes
        tm.begin(STAGE_GROUP);
        launch_group_photons(c, static_cast<const PhotonRay*>(c->phq[in]), &cnt->ph_count[in], c->phq_grouped, st2);
        launches += 3;
        tm.end();
        qin = c->phq_grouped;
      }
      tm.begin(STAGE_TRACE_PHOTON);
      launch_trace_closest(c, reinterpret_cast<const float4*>(qin), &cnt->ph_count[in], c->cap_ph,
                           c->hits_ph, 2, cnt, st2, c->cfg.photon_records);
      tm.end();
      tm.begin(STAGE_PHOTON);
      k_photon<<<capped_blocks(c->cap_ph, kThreads, B), kThreads, 0, st2>>>(s, ip, j, qin, in, c->phq[out], out, c->cfg.photon_records, sl.nv, c->mrec, c->bucket_start, cnt,
                                        accum, split, c->hits_ph, c->oct_nodes, c->oct_state, c->oct,
                                        c->cfg.density_mode == 0, c->mh);
      launches += 3;
      tm.end();
    }
    if (ip.cap_mh > 0) {
      tm.begin(STAGE_MERGE);
      merge_staged(c, ip, sl, accum, split, st2, &launches);
      tm.end();
    }
  }
  return launches;
}

// Records one half of an iteration as a CUDA graph on the private capture
// stream and refreshes `exec` from it (the topology is the same every
// iteration; only kernel parameters change), then launches it on `st`.
// Returns an error, with the capture ended, when any step fails.
template <typename F>
static cudaError_t launch_as_graph(neb_ctx* c, cudaGraphExec_t& exec, cudaStream_t st, F&& enqueue) {
  cudaError_t e = cudaStreamBeginCapture(c->stream_cap, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return e;
  enqueue(c->stream_cap);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(c->stream_cap, &g);
  if (e != cudaSuccess) return e;
  if (exec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(exec, g, &info) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphExecDestroy(exec);
      exec = nullptr;
    }
  }
  if (!exec) e = cudaGraphInstantiate(&exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return e;
  return cudaGraphLaunch(exec, st);
}

cudaError_t run_iteration(neb_ctx* c, int iteration, bool overlap) {
  StageTimer tm(c);  // profiling runs never overlap, so every stage is on c->stream
  long long launches = 0;
  if (!overlap) {
    launches += enqueue_pass1(c, iteration, c->stream, tm);
    launches += enqueue_pass23(c, iteration, c->stream, tm);
    c->launches += launches;
    cudaError_t e = cudaGetLastError();
    tm.collect();
    return e;
  }
  // Pass 1 on stream_hi (the device's highest stream priority, so its blocks
  // are scheduled ahead of the overlapped passes 2-3), passes 2-3 on stream_b.
  // Slot reuse: pass 1 of this iteration waits for passes 2-3 of iteration - 2.
  const int slot = iteration & 1;
  cudaStream_t st = c->stream_hi, st2 = c->stream_b;
  // pass 1 follows whatever the caller enqueued on its stream before this iteration
  cudaEventRecord(c->ev_caller, c->stream);
  cudaStreamWaitEvent(st, c->ev_caller, 0);
  // one half as a graph, or enqueued directly if graphs are off or the
  // recording fails (then they stay off for this context)
  auto half = [&](cudaGraphExec_t& exec, cudaStream_t to, auto enqueue) {
    if (c->use_graphs) {
      long long n = 0;
      cudaError_t e = launch_as_graph(c, exec, to, [&](cudaStream_t cs) { n = enqueue(cs); });
      if (e == cudaSuccess) {
        launches += n;
        return;
      }
      cudaGetLastError();
      c->use_graphs = false;
    }
    launches += enqueue(to);
  };
  cudaStreamWaitEvent(st, c->ev_pass23[slot], 0);
  half(c->graph_pass1[slot], st, [&](cudaStream_t cs) { return enqueue_pass1(c, iteration, cs, tm); });
  cudaEventRecord(c->ev_pass1[slot], st);
  cudaStreamWaitEvent(st2, c->ev_pass1[slot], 0);
  half(c->graph_pass23[slot], st2, [&](cudaStream_t cs) { return enqueue_pass23(c, iteration, cs, tm); });
  cudaEventRecord(c->ev_pass23[slot], st2);
  c->launches += launches;
  return cudaGetLastError();
}

cudaError_t launch_sum_halves(const double* accum, int P, double* out, cudaStream_t st) {
  const int n = 3 * P;
  k_sum_halves<<<(n + 255) / 256, 256, 0, st>>>(accum, n, out);
  return cudaGetLastError();
}

cudaError_t launch_error_sums(const double* accum, int P, int n_even, int n_odd, double* out, cudaStream_t st) {
  cudaMemsetAsync(out, 0, 2 * sizeof(double), st);
  k_error_sums<<<capped_blocks(P, 256, 152 * 4), 256, 0, st>>>(accum, P, n_even, n_odd, out);
  return cudaGetLastError();
}

cudaError_t launch_resolve(const double* accum, int P, int iterations, float* out, cudaStream_t st) {
  int n = P * 3;
  double inv = iterations > 0 ? 1.0 / iterations : 0.0;
  k_resolve<<<(n + 255) / 256, 256, 0, st>>>(accum, n, inv, out);
  return cudaGetLastError();
}

cudaError_t launch_read_rho(neb_ctx* c, float* d_out) {
  const IterSlot& sl = c->slots[c->iteration & 1];  // slot of the last iteration
  k_fill<<<grid_blocks(c), 256, 0, c->stream>>>(d_out, (size_t)c->P * (c->D - 1), -1.0f);  // no NEE vertex
  k_read_rho<<<grid_blocks(c), 256, 0, c->stream>>>(sl.nv, sl.cnt, c->D, c->cap_nee, d_out);
  return cudaGetLastError();
}

}  // namespace neb
