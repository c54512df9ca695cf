/*
 * sc_oracle.c -- plain, slow FP64 CPU oracle of the spectral glass path/light tracer.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may load this library.  It shares no code, header or table with the CUDA
 * library: the two agree only through the scene arrays (float32 world-space triangles)
 * and the published definitions restated below.
 *
 * What it computes.  SuperCaustics (arXiv 2107.11008) renders glass with refraction,
 * reflection, dispersion and caustics (Abstract; Sec. III) and emits pixel-aligned
 * ground truth: depth normalised by a 10 m range (Sec. III-D "Depth Ground Truth"),
 * world- and camera-space normals (Sec. III-D "Surface Normals Ground Truth"), object
 * masks (Sec. III-D "Object Mask Ground Truth") and the caustic mask defined as the
 * luminance difference between renders with and without caustics (Sec. III-D "Local &
 * Non-local Caustics Mask").  The paper's renderer is an engine (Sec. III, NvRTX UE4), so
 * every transport detail below is a stated reading, written out step by step:
 *
 *   RNG        Philox4x32-10 (Salmon et al., SC'11): key = seed, counter = (c0,c1,c2,
 *              tag | scene<<8); u = (x>>8) * 2^-24; an index choice j = (x>>8)*N >> 24.
 *   camera     pinhole, box pixel filter (uniform jitter), y = 0 at the top.
 *   spectrum   B bins over 400-700 nm at bin centres, Cauchy n = A + B/lambda^2 (um);
 *              RGB weight of a bin = linear sRGB of the CIE 1931 fit of Wyman, Sloan and
 *              Shirley (JCGT 2013, multi-lobe), normalised per channel to mean 1 over bins;
 *              B = 1 means no dispersion (n = A, weight 1).
 *   dielectric exact unpolarised Fresnel, Snell refraction, total internal reflection,
 *              reflect iff u < R, throughput unchanged.  Glass variants of Sec. III-C (colour,
 *              roughness): Beer-Lambert absorption over each segment inside the glass, and a
 *              rough dielectric (Walter et al. 2007, GGX) when the material's roughness > 0.
 *   wavelength jitter  optionally lambda = 400 + 300 u from the bin draw (continuous spectrum).
 *   diffuse    Lambert; next-event estimation to one uniformly chosen light (glass blocks
 *              shadow rays); cosine-weighted bounce in the Duff et al. (JCGT 2017) frame.
 *   camera path  emitter radiance is counted only along purely specular prefixes.
 *   light path   emitted from a light, traced through glass, splatted at its first
 *              diffuse vertex after at least one specular event (the caustic, L S+ D E).
 *
 * Every floating-point step is FP64.  Along the way the oracle records how close each
 * discrete decision (which triangle, reflect or refract, visible or not, which pixel)
 * came to flipping; a path with any margin below the tolerances is "ambiguous" and is
 * excluded from bit-exact comparison with an FP32 implementation.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORC_API __attribute__((visibility("default")))

enum { MAT_DIFFUSE = 0, MAT_DIELECTRIC = 1, MAT_EMISSIVE = 2 };
enum { LIGHT_POINT = 0, LIGHT_RECT = 1, LIGHT_DISK = 2 };
enum { FLAG_FORCE_TRANSMIT = 1, FLAG_SPLAT_DIRECT = 2, FLAG_EMITTER_AFTER_DS = 4, FLAG_WAVELENGTH_JITTER = 8 };
enum {
  AMB_EDGE = 1, AMB_TGAP = 2, AMB_GRAZE = 4, AMB_FRESNEL = 8, AMB_TIR = 16,
  AMB_SHADOW = 32, AMB_SPLAT = 64, AMB_CHECKER = 128, AMB_FIXUP = 256, AMB_SENSITIVE = 512
};
enum { EV_MISS = 0xFFFFFFFFu, EV_REFLECT = 1, EV_REFRACT = 2, EV_LIT = 3, EV_UNLIT = 4, EV_FIXUP = 7, EV_KILL = 9 };

static const double PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------------------------ */
/* small vector algebra                                                                        */
/* ------------------------------------------------------------------------------------------ */
typedef struct { double x, y, z; } v3;
static v3 V(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 add(v3 a, v3 b) { return V(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return V(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 mul(v3 a, double s) { return V(a.x * s, a.y * s, a.z * s); }
static v3 hadamard(v3 a, v3 b) { return V(a.x * b.x, a.y * b.y, a.z * b.z); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b) { return V(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
static double len(v3 a) { return sqrt(dot(a, a)); }
static v3 normalize(v3 a) { return mul(a, 1.0 / len(a)); }
static double maxabs(v3 a) { return fmax(fabs(a.x), fmax(fabs(a.y), fabs(a.z))); }
static double comp(v3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel Random Numbers: As Easy as 1, 2, 3")  */
/* ------------------------------------------------------------------------------------------ */
static void philox(const uint32_t ctr_in[4], uint32_t k0, uint32_t k1, uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

ORC_API void orc_philox(const uint32_t *ctr, uint64_t key, int64_t n, uint32_t *out) {
  for (int64_t i = 0; i < n; ++i) philox(ctr + 4 * i, (uint32_t)key, (uint32_t)(key >> 32), out + 4 * i);
}

static void draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t tag, uint32_t scene,
                 uint32_t out[4]) {
  uint32_t c[4] = {c0, c1, c2, tag | (scene << 8)};
  philox(c, (uint32_t)seed, (uint32_t)(seed >> 32), out);
}
static double u01(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }
/* index in [0, n): exact integer form of floor(u * n) */
static int choose(uint32_t x, int n) { return (int)(((uint64_t)(x >> 8) * (uint64_t)n) >> 24); }

/* ------------------------------------------------------------------------------------------ */
/* spectrum                                                                                    */
/* ------------------------------------------------------------------------------------------ */
/* piecewise Gaussian of the Wyman-Sloan-Shirley fit: width s1 left of the mean, s2 right */
static double g_lobe(double lam, double mu, double s1, double s2) {
  double s = lam < mu ? s1 : s2;
  double t = (lam - mu) / s;
  return exp(-0.5 * t * t);
}
static v3 cie_xyz(double lam) {
  double x = 1.056 * g_lobe(lam, 599.8, 37.9, 31.0) + 0.362 * g_lobe(lam, 442.0, 16.0, 26.7) -
             0.065 * g_lobe(lam, 501.1, 20.4, 26.2);
  double y = 0.821 * g_lobe(lam, 568.8, 46.9, 40.5) + 0.286 * g_lobe(lam, 530.9, 16.3, 31.1);
  double z = 1.217 * g_lobe(lam, 437.0, 11.8, 36.0) + 0.681 * g_lobe(lam, 459.0, 26.0, 13.8);
  return V(x, y, z);
}
/* CIE XYZ -> linear sRGB (D65), IEC 61966-2-1 */
static v3 xyz_to_rgb(v3 c) {
  return V(3.2404542 * c.x - 1.5371385 * c.y - 0.4985314 * c.z,
           -0.9692660 * c.x + 1.8760108 * c.y + 0.0415560 * c.z,
           0.0556434 * c.x - 0.2040259 * c.y + 1.0572252 * c.z);
}
ORC_API void orc_cie_xyz(double lam, double *out) {
  v3 c = cie_xyz(lam);
  out[0] = c.x; out[1] = c.y; out[2] = c.z;
}
ORC_API void orc_xyz_to_rgb(const double *in, double *out) {
  v3 c = xyz_to_rgb(V(in[0], in[1], in[2]));
  out[0] = c.x; out[1] = c.y; out[2] = c.z;
}
static double bin_lambda(int b, int nbins) { return 400.0 + (b + 0.5) * 300.0 / nbins; }

ORC_API void orc_spectral_weights(int nbins, double *w /* nbins*3 */, double *lambda /* nbins */) {
  if (nbins <= 1) { w[0] = w[1] = w[2] = 1.0; if (lambda) lambda[0] = 550.0; return; }
  v3 mean = V(0, 0, 0);
  for (int b = 0; b < nbins; ++b) {
    v3 c = xyz_to_rgb(cie_xyz(bin_lambda(b, nbins)));
    w[3 * b] = c.x; w[3 * b + 1] = c.y; w[3 * b + 2] = c.z;
    mean = add(mean, mul(c, 1.0 / nbins));
    if (lambda) lambda[b] = bin_lambda(b, nbins);
  }
  for (int b = 0; b < nbins; ++b) { w[3 * b] /= mean.x; w[3 * b + 1] /= mean.y; w[3 * b + 2] /= mean.z; }
}

/* Cauchy index at wavelength lam (nm); one bin means no dispersion */
static double cauchy_at(double A, double B, double lam, int nbins) {
  if (nbins <= 1) return A;
  double lum = lam * 1e-3;
  return A + B / (lum * lum);
}

/* Sub-bin wavelength jitter (Sec. III-C varies the glass; a reading of how a renderer samples the
 * spectrum continuously): the bin draw u gives lam = 400 + 300 u, uniform over 400-700 nm, whose
 * bin is still floor(u B).  Its RGB weight is the CIE fit's linear sRGB at lam divided per channel
 * by the fit's mean over 400-700 nm, so that a flat spectrum stays white in expectation.  The mean
 * is the composite Simpson rule with 6000 intervals. */
static v3 g_jitter_mean;
static pthread_once_t g_jitter_once = PTHREAD_ONCE_INIT;
static void jitter_mean_init(void) {
  const int n = 6000;
  const double h = 300.0 / n;
  v3 acc = add(xyz_to_rgb(cie_xyz(400.0)), xyz_to_rgb(cie_xyz(700.0)));
  for (int i = 1; i < n; ++i) acc = add(acc, mul(xyz_to_rgb(cie_xyz(400.0 + i * h)), (i & 1) ? 4.0 : 2.0));
  g_jitter_mean = mul(acc, h / 3.0 / 300.0);
}
static v3 jitter_mean(void) {
  pthread_once(&g_jitter_once, jitter_mean_init);
  return g_jitter_mean;
}
ORC_API void orc_jitter_mean(double *out) {
  v3 m = jitter_mean();
  out[0] = m.x; out[1] = m.y; out[2] = m.z;
}

/* the wavelength of a path and its RGB weight, from the bin draw x */
typedef struct { int bin; double lam; v3 w; } spec_sample;
static spec_sample spectral_sample(uint32_t x, int nbins, int flags, const double *wts) {
  spec_sample sp;
  sp.bin = choose(x, nbins > 0 ? nbins : 1);
  if (nbins <= 1) { sp.lam = 550.0; sp.w = V(1, 1, 1); return sp; }
  if (flags & FLAG_WAVELENGTH_JITTER) {
    sp.lam = 400.0 + 300.0 * u01(x);
    v3 c = xyz_to_rgb(cie_xyz(sp.lam)), m = jitter_mean();
    sp.w = V(c.x / m.x, c.y / m.y, c.z / m.z);
  } else {
    sp.lam = bin_lambda(sp.bin, nbins);
    sp.w = V(wts[3 * sp.bin], wts[3 * sp.bin + 1], wts[3 * sp.bin + 2]);
  }
  return sp;
}

/* ------------------------------------------------------------------------------------------ */
/* optics primitives                                                                           */
/* ------------------------------------------------------------------------------------------ */
/* exact unpolarised Fresnel reflectance (average of s and p), Hecht "Optics" Sec. 4.6 */
static double fresnel(double cos_i, double cos_t, double n_i, double n_t) {
  double rs = (n_i * cos_i - n_t * cos_t) / (n_i * cos_i + n_t * cos_t);
  double rp = (n_i * cos_t - n_t * cos_i) / (n_i * cos_t + n_t * cos_i);
  return 0.5 * (rs * rs + rp * rp);
}
/* reflectance for an incidence cosine; total internal reflection gives 1 */
ORC_API double orc_fresnel(double cos_i, double n_i, double n_t) {
  double eta = n_i / n_t;
  double k = 1.0 - eta * eta * (1.0 - cos_i * cos_i);
  if (k < 0) return 1.0;
  return fresnel(cos_i, sqrt(k), n_i, n_t);
}
/* Snell refraction of unit d through unit normal n facing d's origin side; returns 0 on TIR */
static int refract_dir(v3 d, v3 n, double eta, v3 *out, double *k_out) {
  double cos_i = -dot(d, n);
  double k = 1.0 - eta * eta * (1.0 - cos_i * cos_i);
  if (k_out) *k_out = k;
  if (k < 0) return 0;
  *out = normalize(add(mul(d, eta), mul(n, eta * cos_i - sqrt(k))));
  return 1;
}
ORC_API int orc_refract(const double *d, const double *n, double eta, double *out) {
  v3 o;
  if (!refract_dir(V(d[0], d[1], d[2]), V(n[0], n[1], n[2]), eta, &o, NULL)) return 0;
  out[0] = o.x; out[1] = o.y; out[2] = o.z;
  return 1;
}
/* orthonormal basis around unit n (Duff, Burgess, Christensen, Hery, Kensler, Liani, Villemin,
 * "Building an Orthonormal Basis, Revisited", JCGT 2017) */
static void onb(v3 n, v3 *t1, v3 *t2) {
  double sign = copysign(1.0, n.z);
  double a = -1.0 / (sign + n.z);
  double b = n.x * n.y * a;
  *t1 = V(1.0 + sign * n.x * n.x * a, sign * b, -sign * n.x);
  *t2 = V(b, sign + n.y * n.y * a, -n.y);
}
static v3 cosine_dir(v3 n, double u1, double u2) {
  v3 t1, t2;
  onb(n, &t1, &t2);
  double r = sqrt(u1), phi = 2.0 * PI * u2;
  return normalize(add(add(mul(t1, r * cos(phi)), mul(t2, r * sin(phi))), mul(n, sqrt(fmax(0.0, 1.0 - u1)))));
}

/* ------------------------------------------------------------------------------------------ */
/* scene                                                                                       */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  int kind; v3 a1, a2; double checker, A, B; v3 emission;
  v3 absorb;     /* dielectric: Beer-Lambert absorption coefficient per metre (RGB) */
  double alpha;  /* dielectric: GGX roughness (0 = smooth) */
} material;
typedef struct {
  int kind; v3 p, u, v, power; double radius;
} light;
typedef struct {
  double lo[3], hi[3];
  int left, right; /* children (internal) or -1 */
  int first, count; /* leaf range in tri_order */
} bnode;
typedef struct {
  int nt;
  v3 *v; /* nt*3 */
  v3 *n; /* nt*3 */
  double *uv; /* nt*6 */
  int *smooth, *mat, *obj;
  double *alt; /* nt*3 altitudes h0,h1,h2 */
  v3 *ng; /* unit geometric normals */
  int nmat, nlights;
  material *mats;
  light *lights;
  v3 eye, look, up, f, r, u;
  double vfov, th, aspect;
  int W, H;
  v3 env;
  bnode *nodes;
  int nnodes;
  int *tri_order;
  double box_pad;
} scene;

typedef struct {
  double pos;    /* edge / near-miss / checker distance, relative to max(1,|p|inf) */
  double t;      /* relative gap between the two closest hits */
  double cosg;   /* |cos| against the geometric normal, |u - R| style direction margins */
  double fres;   /* |u - R| of a Fresnel draw */
  double tir;    /* |cos_t^2| near total internal reflection */
  double px;     /* splat distance to a pixel border, in pixels */
  double growth; /* each specular event before a decision multiplies its tolerance by this */
  double sens_delta; /* relative size of the ray perturbations of the sensitivity re-traces (0 = off) */
  double sens_rel;   /* a re-trace moving the radiance by more than this (relative) flags the path */
} tolerances;

static const tolerances DEFAULT_TOL = {2e-5, 1e-5, 1e-4, 1e-4, 1e-5, 1e-4, 1.0, 0.0, 1e-4};

/* near misses are tracked inside this window (relative), wider than any tolerance */
#define NM_WIN 1e-3
#define T_WIN 1e-3

static int cmp_axis;
static const double *cmp_cent;
static int cmp_idx(const void *a, const void *b) {
  double x = cmp_cent[3 * (*(const int *)a) + cmp_axis], y = cmp_cent[3 * (*(const int *)b) + cmp_axis];
  if (x < y) return -1;
  if (x > y) return 1;
  return (*(const int *)a) - (*(const int *)b);
}

/* median-split BVH: split the longest centroid axis at the median, leaves of <= 4 triangles */
static int bvh_build(scene *s, const double *cent, int first, int count) {
  int id = s->nnodes++;
  bnode *nd = &s->nodes[id];
  for (int k = 0; k < 3; ++k) { nd->lo[k] = INFINITY; nd->hi[k] = -INFINITY; }
  double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int i = first; i < first + count; ++i) {
    int t = s->tri_order[i];
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) {
        double c = comp(s->v[3 * t + j], k);
        nd->lo[k] = fmin(nd->lo[k], c); nd->hi[k] = fmax(nd->hi[k], c);
      }
    for (int k = 0; k < 3; ++k) { clo[k] = fmin(clo[k], cent[3 * t + k]); chi[k] = fmax(chi[k], cent[3 * t + k]); }
  }
  for (int k = 0; k < 3; ++k) {
    double pad = s->box_pad * fmax(1.0, fmax(fabs(nd->lo[k]), fabs(nd->hi[k])));
    nd->lo[k] -= pad; nd->hi[k] += pad;
  }
  if (count <= 4) {
    nd->left = nd->right = -1; nd->first = first; nd->count = count;
    return id;
  }
  int axis = 0;
  for (int k = 1; k < 3; ++k) if (chi[k] - clo[k] > chi[axis] - clo[axis]) axis = k;
  cmp_axis = axis; cmp_cent = cent;
  qsort(s->tri_order + first, count, sizeof(int), cmp_idx);
  int half = count / 2;
  int l = bvh_build(s, cent, first, half);
  int r = bvh_build(s, cent, first + half, count - half);
  nd = &s->nodes[id];
  nd->left = l; nd->right = r; nd->first = 0; nd->count = 0;
  return id;
}

ORC_API void *orc_scene_create(int nv, const float *pos, const float *nrm, const float *uv, int nt, const int *idx,
                                const int *tri_obj, int nobj, const int *obj_mat, int nmat, const double *mats,
                                int nlights, const double *lights, const double *cam, int W, int H,
                                const double *env) {
  (void)nv; (void)nobj;
  scene *s = calloc(1, sizeof(scene));
  s->nt = nt;
  s->v = malloc(sizeof(v3) * 3 * (size_t)(nt > 0 ? nt : 1));
  s->n = malloc(sizeof(v3) * 3 * (size_t)(nt > 0 ? nt : 1));
  s->uv = malloc(sizeof(double) * 6 * (size_t)(nt > 0 ? nt : 1));
  s->smooth = malloc(sizeof(int) * (size_t)(nt > 0 ? nt : 1));
  s->mat = malloc(sizeof(int) * (size_t)(nt > 0 ? nt : 1));
  s->obj = malloc(sizeof(int) * (size_t)(nt > 0 ? nt : 1));
  s->alt = malloc(sizeof(double) * 3 * (size_t)(nt > 0 ? nt : 1));
  s->ng = malloc(sizeof(v3) * (size_t)(nt > 0 ? nt : 1));
  for (int t = 0; t < nt; ++t) {
    int sm = 1;
    for (int j = 0; j < 3; ++j) {
      int vi = idx[3 * t + j];
      s->v[3 * t + j] = V(pos[3 * vi], pos[3 * vi + 1], pos[3 * vi + 2]);
      s->n[3 * t + j] = nrm ? V(nrm[3 * vi], nrm[3 * vi + 1], nrm[3 * vi + 2]) : V(0, 0, 0);
      if (s->n[3 * t + j].x == 0 && s->n[3 * t + j].y == 0 && s->n[3 * t + j].z == 0) sm = 0;
      s->uv[6 * t + 2 * j] = uv ? uv[2 * vi] : 0.0;
      s->uv[6 * t + 2 * j + 1] = uv ? uv[2 * vi + 1] : 0.0;
    }
    s->smooth[t] = sm;
    s->obj[t] = tri_obj[t];
    s->mat[t] = obj_mat[tri_obj[t]];
    v3 e1 = sub(s->v[3 * t + 1], s->v[3 * t]), e2 = sub(s->v[3 * t + 2], s->v[3 * t]);
    v3 c = cross(e1, e2);
    double a2 = len(c);
    s->ng[t] = a2 > 0 ? mul(c, 1.0 / a2) : V(0, 0, 0);
    /* altitude from vertex k onto the opposite edge = 2 * area / |opposite edge| */
    double l0 = len(sub(s->v[3 * t + 2], s->v[3 * t + 1]));
    double l1 = len(sub(s->v[3 * t + 2], s->v[3 * t]));
    double l2 = len(sub(s->v[3 * t + 1], s->v[3 * t]));
    s->alt[3 * t] = l0 > 0 ? a2 / l0 : 0; s->alt[3 * t + 1] = l1 > 0 ? a2 / l1 : 0;
    s->alt[3 * t + 2] = l2 > 0 ? a2 / l2 : 0;
  }
  s->nmat = nmat;
  s->mats = calloc((size_t)(nmat > 0 ? nmat : 1), sizeof(material));
  for (int m = 0; m < nmat; ++m) {
    const double *q = mats + 17 * m;
    s->mats[m].kind = (int)q[0];
    s->mats[m].a1 = V(q[1], q[2], q[3]); s->mats[m].a2 = V(q[4], q[5], q[6]);
    s->mats[m].checker = q[7]; s->mats[m].A = q[8]; s->mats[m].B = q[9];
    s->mats[m].emission = V(q[10], q[11], q[12]);
    s->mats[m].absorb = V(q[13], q[14], q[15]);
    s->mats[m].alpha = q[16];
  }
  s->nlights = nlights;
  s->lights = calloc((size_t)(nlights > 0 ? nlights : 1), sizeof(light));
  for (int l = 0; l < nlights; ++l) {
    const double *q = lights + 14 * l;
    s->lights[l].kind = (int)q[0];
    s->lights[l].p = V(q[1], q[2], q[3]); s->lights[l].u = V(q[4], q[5], q[6]);
    s->lights[l].v = V(q[7], q[8], q[9]); s->lights[l].power = V(q[10], q[11], q[12]);
    s->lights[l].radius = q[13];
  }
  s->eye = V(cam[0], cam[1], cam[2]); s->look = V(cam[3], cam[4], cam[5]); s->up = V(cam[6], cam[7], cam[8]);
  s->vfov = cam[9];
  s->f = normalize(sub(s->look, s->eye));
  s->r = normalize(cross(s->f, s->up));
  s->u = cross(s->r, s->f);
  s->th = tan(0.5 * s->vfov * PI / 180.0);
  s->W = W; s->H = H; s->aspect = (double)W / (double)H;
  s->env = V(env[0], env[1], env[2]);
  /* BVH with boxes padded so that near misses are still visited */
  s->box_pad = 2.0 * NM_WIN;
  s->nodes = malloc(sizeof(bnode) * (size_t)(2 * (nt > 0 ? nt : 1)));
  s->tri_order = malloc(sizeof(int) * (size_t)(nt > 0 ? nt : 1));
  double *cent = malloc(sizeof(double) * 3 * (size_t)(nt > 0 ? nt : 1));
  for (int t = 0; t < nt; ++t) {
    s->tri_order[t] = t;
    v3 c = mul(add(add(s->v[3 * t], s->v[3 * t + 1]), s->v[3 * t + 2]), 1.0 / 3.0);
    cent[3 * t] = c.x; cent[3 * t + 1] = c.y; cent[3 * t + 2] = c.z;
  }
  s->nnodes = 0;
  if (nt > 0) bvh_build(s, cent, 0, nt);
  free(cent);
  return s;
}

ORC_API void orc_scene_destroy(void *p) {
  scene *s = p;
  if (!s) return;
  free(s->v); free(s->n); free(s->uv); free(s->smooth); free(s->mat); free(s->obj); free(s->alt); free(s->ng);
  free(s->mats); free(s->lights); free(s->nodes); free(s->tri_order);
  free(s);
}

/* ------------------------------------------------------------------------------------------ */
/* decision margins: how far each discrete decision of a path was from flipping                */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  const tolerances *tol;
  int nspec;         /* specular events so far */
  int amb;           /* flags of decisions inside their (grown) tolerance */
  double min_ratio;  /* smallest margin / base tolerance over the path */
  int ratio_nspec;   /* specular events before that decision */
  int ratio_kind;    /* its flag */
  double kmin[9];    /* smallest margin / base tolerance per decision kind (bit index of the flag) */
  int knspec[9];     /* specular events before it */
} actx;

static void actx_init(actx *a, const tolerances *tol) {
  a->tol = tol; a->nspec = 0; a->amb = 0; a->min_ratio = INFINITY; a->ratio_nspec = 0; a->ratio_kind = 0;
  for (int i = 0; i < 9; ++i) { a->kmin[i] = INFINITY; a->knspec[i] = 0; }
}
/* margin m against base tolerance b: flagged when m < b * growth^nspec */
static void note(actx *a, double m, double b, int flag) {
  double r = m / b;
  if (r < a->min_ratio) { a->min_ratio = r; a->ratio_nspec = a->nspec; a->ratio_kind = flag; }
  int k = __builtin_ctz((unsigned)flag);
  if (r < a->kmin[k]) { a->kmin[k] = r; a->knspec[k] = a->nspec; }
  if (r < pow(a->tol->growth, a->nspec)) a->amb |= flag;
}

/* ------------------------------------------------------------------------------------------ */
/* ray / triangle (Moller-Trumbore 1997, FP64, inclusive edges)                                */
/* ------------------------------------------------------------------------------------------ */
typedef struct { v3 o, d; } ray;
typedef struct {
  int tri;        /* -1 = miss */
  double t, b1, b2;
  double m_edge;  /* distance (world units) to flipping the hit triangle: own edges, closer near misses */
  double m_tgap;  /* relative gap to the second closest hit */
  double scale;   /* max(1, |p|inf) at the decision point */
} hit;

/* plane intersection: returns 0 if the ray is parallel to the triangle's plane */
static int mt(const scene *s, int t, ray r, double *tt, double *u, double *v) {
  v3 v0 = s->v[3 * t], e1 = sub(s->v[3 * t + 1], v0), e2 = sub(s->v[3 * t + 2], v0);
  v3 pv = cross(r.d, e2);
  double det = dot(e1, pv);
  if (det == 0.0) return 0;
  double inv = 1.0 / det;
  v3 tv = sub(r.o, v0);
  *u = dot(tv, pv) * inv;
  v3 qv = cross(tv, e1);
  *v = dot(r.d, qv) * inv;
  *tt = dot(e2, qv) * inv;
  return 1;
}
/* signed distance (world units) from the plane hit point to the nearest edge; < 0 outside */
static double edge_margin(const scene *s, int t, double u, double v) {
  double d0 = (1.0 - u - v) * s->alt[3 * t], d1 = u * s->alt[3 * t + 1], d2 = v * s->alt[3 * t + 2];
  return fmin(d0, fmin(d1, d2));
}

static int box_hit(const bnode *nd, ray r, double tmax) {
  double t0 = 0.0, t1 = tmax;
  for (int k = 0; k < 3; ++k) {
    double o = comp(r.o, k), d = comp(r.d, k);
    if (d == 0.0) {
      if (o < nd->lo[k] || o > nd->hi[k]) return 0;
      continue;
    }
    double a = (nd->lo[k] - o) / d, b = (nd->hi[k] - o) / d;
    if (a > b) { double x = a; a = b; b = x; }
    t0 = fmax(t0, a); t1 = fmin(t1, b);
    if (t0 > t1) return 0;
  }
  return 1;
}

#define NEAR_MAX 16
typedef struct {
  int best; double bt, bu, bv, bmargin, bscale;
  double t2;                        /* second closest hit */
  int nn;                           /* near misses kept (closest in t) */
  double nt[NEAR_MAX], nd[NEAR_MAX], ns[NEAR_MAX];
} closest_state;

static void closest_test(const scene *s, int t, ray r, closest_state *cs) {
  double tt, u, v;
  if (!mt(s, t, r, &tt, &u, &v)) return;
  if (!(tt > 0.0)) return;
  v3 p = add(r.o, mul(r.d, tt));
  double m = edge_margin(s, t, u, v);
  double scale = fmax(1.0, maxabs(p));
  if (m >= 0.0) {
    if (tt < cs->bt || (tt == cs->bt && t < cs->best)) {
      if (cs->best >= 0) cs->t2 = fmin(cs->t2, cs->bt);
      cs->best = t; cs->bt = tt; cs->bu = u; cs->bv = v; cs->bmargin = m; cs->bscale = scale;
    } else {
      cs->t2 = fmin(cs->t2, tt);
    }
  } else if (-m < NM_WIN * scale) {
    /* keep the near misses with the smallest t */
    int slot = cs->nn < NEAR_MAX ? cs->nn++ : -1;
    if (slot < 0) {
      int worst = 0;
      for (int i = 1; i < NEAR_MAX; ++i) if (cs->nt[i] > cs->nt[worst]) worst = i;
      if (cs->nt[worst] <= tt) return;
      slot = worst;
    }
    cs->nt[slot] = tt; cs->nd[slot] = -m; cs->ns[slot] = scale;
  }
}

static hit closest(const scene *s, ray r, int brute) {
  closest_state cs;
  cs.best = -1; cs.bt = INFINITY; cs.bu = cs.bv = cs.bmargin = 0; cs.bscale = 1; cs.t2 = INFINITY; cs.nn = 0;
  if (brute || s->nnodes == 0) {
    for (int t = 0; t < s->nt; ++t) closest_test(s, t, r, &cs);
  } else {
    int stack[128], sp = 0;
    stack[sp++] = 0;
    while (sp) {
      const bnode *nd = &s->nodes[stack[--sp]];
      if (!box_hit(nd, r, cs.bt * (1.0 + 4.0 * T_WIN) + 1e-12)) continue;
      if (nd->left < 0) {
        for (int i = nd->first; i < nd->first + nd->count; ++i) closest_test(s, s->tri_order[i], r, &cs);
      } else {
        stack[sp++] = nd->left;
        stack[sp++] = nd->right;
      }
    }
  }
  hit h;
  h.tri = cs.best; h.t = cs.bt; h.b1 = cs.bu; h.b2 = cs.bv;
  h.m_edge = INFINITY; h.m_tgap = INFINITY; h.scale = cs.bscale;
  if (cs.best >= 0) {
    h.m_edge = cs.bmargin;
    for (int i = 0; i < cs.nn; ++i)
      if (cs.nt[i] <= cs.bt * (1.0 + T_WIN)) h.m_edge = fmin(h.m_edge, cs.nd[i]);
    if (cs.t2 < INFINITY) h.m_tgap = (cs.t2 - cs.bt) / cs.bt;
  } else {
    for (int i = 0; i < cs.nn; ++i)
      if (cs.nd[i] < h.m_edge) { h.m_edge = cs.nd[i]; h.scale = cs.ns[i]; }
  }
  return h;
}

/* closest hit plus its margins noted in the path context */
static hit closest_noted(const scene *s, ray r, int brute, actx *a) {
  hit h = closest(s, r, brute);
  const tolerances *tol = a->tol;
  note(a, h.m_edge, tol->pos * h.scale, AMB_EDGE);
  note(a, h.m_tgap, tol->t, AMB_TGAP);
  return h;
}

/* any hit with t in (0, tmax); *margin = world distance to flipping the answer (inf if robust) */
typedef struct {
  int hitany, robust;
  double margin;  /* relative to scale */
  double tgap;    /* relative distance of a hit / near miss to tmax */
} occ_state;

static void any_test(const scene *s, int t, ray r, double tmax, occ_state *os) {
  double tt, u, v;
  if (!mt(s, t, r, &tt, &u, &v)) return;
  if (!(tt > 0.0)) return;
  if (tt >= tmax * (1.0 + T_WIN)) return;
  v3 p = add(r.o, mul(r.d, tt));
  double m = edge_margin(s, t, u, v);
  double scale = fmax(1.0, maxabs(p));
  double gap = fabs(tt - tmax) / tmax;
  if (m >= 0.0 && tt < tmax) {
    os->hitany = 1;
    if (m >= NM_WIN * scale && gap >= T_WIN) { os->robust = 1; return; }
  }
  if (fabs(m) < NM_WIN * scale) os->margin = fmin(os->margin, fabs(m) / scale);
  if (m >= 0.0 || fabs(m) < NM_WIN * scale) os->tgap = fmin(os->tgap, gap);
}

static int occluded_m(const scene *s, ray r, double tmax, int brute, double *margin, double *tgap) {
  occ_state os = {0, 0, INFINITY, INFINITY};
  if (brute || s->nnodes == 0) {
    for (int t = 0; t < s->nt && !os.robust; ++t) any_test(s, t, r, tmax, &os);
  } else {
    int stack[128], sp = 0;
    stack[sp++] = 0;
    while (sp && !os.robust) {
      const bnode *nd = &s->nodes[stack[--sp]];
      if (!box_hit(nd, r, tmax * (1.0 + 4.0 * T_WIN))) continue;
      if (nd->left < 0) {
        for (int i = nd->first; i < nd->first + nd->count && !os.robust; ++i) any_test(s, s->tri_order[i], r, tmax, &os);
      } else {
        stack[sp++] = nd->left;
        stack[sp++] = nd->right;
      }
    }
  }
  *margin = os.robust ? INFINITY : os.margin;
  *tgap = os.robust ? INFINITY : os.tgap;
  return os.hitany;
}

static int occluded_noted(const scene *s, ray r, double tmax, int brute, actx *a) {
  double m, g;
  int occ = occluded_m(s, r, tmax, brute, &m, &g);
  note(a, m, a->tol->pos, AMB_SHADOW);
  note(a, g, a->tol->t, 32);
  return occ;
}

ORC_API void orc_intersect(void *sp, int64_t n, const double *rays, int brute, double *t_out, int *tri_out,
                           double *b_out, int *amb_out) {
  const scene *s = sp;
  for (int64_t i = 0; i < n; ++i) {
    ray r = {V(rays[6 * i], rays[6 * i + 1], rays[6 * i + 2]), V(rays[6 * i + 3], rays[6 * i + 4], rays[6 * i + 5])};
    actx a;
    actx_init(&a, &DEFAULT_TOL);
    hit h = closest_noted(s, r, brute, &a);
    t_out[i] = h.t; tri_out[i] = h.tri;
    if (b_out) { b_out[2 * i] = h.b1; b_out[2 * i + 1] = h.b2; }
    if (amb_out) amb_out[i] = a.amb;
  }
}

ORC_API void orc_occluded(void *sp, int64_t n, const double *rays, const double *tmax, int brute, int *occ,
                          int *amb) {
  const scene *s = sp;
  for (int64_t i = 0; i < n; ++i) {
    ray r = {V(rays[6 * i], rays[6 * i + 1], rays[6 * i + 2]), V(rays[6 * i + 3], rays[6 * i + 4], rays[6 * i + 5])};
    actx a;
    actx_init(&a, &DEFAULT_TOL);
    occ[i] = occluded_noted(s, r, tmax[i], brute, &a);
    if (amb) amb[i] = a.amb;
  }
}

/* ------------------------------------------------------------------------------------------ */
/* surface interaction                                                                         */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  v3 p, ng, ns;   /* point, unit geometric normal (winding), unit shading normal on ng's side */
  v3 ngf, nsf;    /* both oriented toward the side the ray came from */
  double cosg;    /* dot(d, ng) */
  int mat;
  double u, v;    /* barycentrics of v1, v2 */
} surf;

static surf interact(const scene *s, ray r, hit h) {
  surf f;
  int t = h.tri;
  double b0 = 1.0 - h.b1 - h.b2;
  f.u = h.b1; f.v = h.b2;
  f.p = add(add(mul(s->v[3 * t], b0), mul(s->v[3 * t + 1], h.b1)), mul(s->v[3 * t + 2], h.b2));
  f.ng = s->ng[t];
  if (s->smooth[t]) {
    f.ns = normalize(add(add(mul(s->n[3 * t], b0), mul(s->n[3 * t + 1], h.b1)), mul(s->n[3 * t + 2], h.b2)));
    if (dot(f.ns, f.ng) < 0) f.ns = mul(f.ns, -1.0);
  } else {
    f.ns = f.ng;
  }
  f.cosg = dot(r.d, f.ng);
  double side = f.cosg < 0 ? 1.0 : -1.0;
  f.ngf = mul(f.ng, side);
  f.nsf = mul(f.ns, side);
  f.mat = s->mats ? s->mat[t] : 0;
  return f;
}

static double eps_of(v3 p) { return 1e-4 * fmax(1.0, maxabs(p)); }
static v3 offset_along(v3 p, v3 ng, v3 dir) {
  double sgn = dot(dir, ng) >= 0 ? 1.0 : -1.0;
  return add(p, mul(ng, sgn * eps_of(p)));
}

static v3 albedo_at(const scene *s, int tri, const surf *f, actx *a) {
  const material *m = &s->mats[f->mat];
  if (m->checker <= 0) return m->a1;
  double b0 = 1.0 - f->u - f->v;
  const double *q = s->uv + 6 * tri;
  double su = (b0 * q[0] + f->u * q[2] + f->v * q[4]) * m->checker;
  double sv = (b0 * q[1] + f->u * q[3] + f->v * q[5]) * m->checker;
  double fu = floor(su), fv = floor(sv);
  if (a) {
    /* distance to the nearest cell border, in world units of the surface */
    double du = fmin(su - fu, fu + 1 - su) / m->checker, dv = fmin(sv - fv, fv + 1 - sv) / m->checker;
    note(a, fmin(du, dv), a->tol->pos * fmax(1.0, maxabs(f->p)), AMB_CHECKER);
  }
  long parity = ((long)fu + (long)fv) & 1;
  return parity ? m->a2 : m->a1;
}

/* dielectric scatter; returns the new direction and whether it reflected */
static v3 dielectric(const surf *f, v3 d, double n_lambda, double u0, int flags, int *reflected, int *fixup,
                     actx *a) {
  int entering = f->cosg < 0;
  double n_i = entering ? 1.0 : n_lambda, n_t = entering ? n_lambda : 1.0;
  double eta = n_i / n_t;
  v3 out = d;
  *fixup = 0;
  for (int pass = 0; pass < 2; ++pass) {
    v3 n = pass == 0 ? f->nsf : f->ngf;
    double cos_i = -dot(d, n);
    if (pass == 0) note(a, fabs(cos_i), a->tol->cosg, AMB_FIXUP);
    if (pass == 0 && cos_i <= 0) { *fixup = 1; continue; }
    double k = 1.0 - eta * eta * (1.0 - cos_i * cos_i);
    note(a, fabs(k), a->tol->tir, AMB_TIR);
    double R = 1.0;
    if (k >= 0) {
      R = fresnel(cos_i, sqrt(k), n_i, n_t);
      if (!(flags & FLAG_FORCE_TRANSMIT)) note(a, fabs(u0 - R), a->tol->fres, AMB_FRESNEL);
    }
    int refl = (k < 0) || (!(flags & FLAG_FORCE_TRANSMIT) && u0 < R);
    if (refl) out = normalize(add(d, mul(n, 2.0 * cos_i)));
    else out = normalize(add(mul(d, eta), mul(n, eta * cos_i - sqrt(k))));
    *reflected = refl;
    double side = dot(out, f->ngf);
    note(a, fabs(side), a->tol->cosg, AMB_FIXUP);
    int ok = refl ? side > 0 : side < 0;
    if (ok || pass == 1) break;
    *fixup = 1;
  }
  return out;
}

/* Smith masking term of GGX for a direction at cosine cos_v to the macro normal (Walter et al.
 * 2007, eq. 34; the sign condition on v.m is checked by the caller) */
static double ggx_g1(double cos_v, double alpha) {
  double c2 = cos_v * cos_v;
  double tan2 = (1.0 - c2) / c2;
  return 2.0 / (1.0 + sqrt(1.0 + alpha * alpha * tan2));
}

/* Rough dielectric (Walter, Marschner, Li, Torrance, "Microfacet Models for Refraction through
 * Rough Surfaces", EGSR 2007), GGX distribution of width alpha.  Macro normal n = the shading
 * normal facing the ray (the geometric one if the shading normal faces away).  A microfacet normal
 * m is drawn with density D(m) |m.n|: tan^2(theta_m) = alpha^2 u1 / (1 - u1), phi_m = 2 pi u2 in the
 * Duff et al. frame of n.  Reflection or refraction about m is chosen as for a smooth surface with
 * the Fresnel reflectance at m (u0 < F), and the throughput is multiplied by the estimator weight
 * of that sampling, |i.m| G1(i) G1(o) / (|i.n| |m.n|) (Walter et al. eq. 41; i = -d the direction
 * back to the ray's origin, o the new direction).  Returns 0 (the path ends) when m faces away
 * from i or o leaves on the wrong side of the macro or the geometric surface. */
static int rough_dielectric(const surf *f, v3 d, double n_lambda, double alpha, double u0, double u1, double u2,
                            int flags, v3 *out, double *weight, int *reflected, int *fixup, actx *a) {
  int entering = f->cosg < 0;
  double n_i = entering ? 1.0 : n_lambda, n_t = entering ? n_lambda : 1.0;
  double eta = n_i / n_t;
  v3 n = f->nsf;
  double cn = -dot(d, n);
  note(a, fabs(cn), a->tol->cosg, AMB_FIXUP);
  *fixup = 0;
  *reflected = 0;
  *weight = 0.0;
  if (!(cn > 0)) {
    n = f->ngf;
    cn = -dot(d, n);
    *fixup = 1;
  }
  v3 t1, t2;
  onb(n, &t1, &t2);
  double tan2 = alpha * alpha * u1 / (1.0 - u1);
  double cm = 1.0 / sqrt(1.0 + tan2), sm = sqrt(fmax(0.0, 1.0 - cm * cm)), phi = 2.0 * PI * u2;
  v3 m = normalize(add(add(mul(t1, sm * cos(phi)), mul(t2, sm * sin(phi))), mul(n, cm)));
  double c = -dot(d, m);
  note(a, fabs(c), a->tol->cosg, AMB_GRAZE);
  if (!(c > 0)) return 0;
  double k = 1.0 - eta * eta * (1.0 - c * c);
  note(a, fabs(k), a->tol->tir, AMB_TIR);
  double R = 1.0;
  if (k >= 0) {
    R = fresnel(c, sqrt(k), n_i, n_t);
    if (!(flags & FLAG_FORCE_TRANSMIT)) note(a, fabs(u0 - R), a->tol->fres, AMB_FRESNEL);
  }
  int refl = (k < 0) || (!(flags & FLAG_FORCE_TRANSMIT) && u0 < R);
  v3 o = refl ? normalize(add(d, mul(m, 2.0 * c))) : normalize(add(mul(d, eta), mul(m, eta * c - sqrt(k))));
  *reflected = refl;
  double sg = dot(o, f->ngf), sn = dot(o, n), om = dot(o, m);
  note(a, fabs(sg), a->tol->cosg, AMB_FIXUP);
  note(a, fabs(sn), a->tol->cosg, AMB_FIXUP);
  if (refl ? !(sg > 0 && sn > 0) : !(sg < 0 && sn < 0)) return 0;
  if (!(om * sn > 0)) return 0;
  *weight = c * ggx_g1(cn, alpha) * ggx_g1(fabs(sn), alpha) / (cn * cm);
  *out = o;
  return 1;
}

/* one rough scatter for the pins: d, ns, ng unit; the surface faces d's origin as for a hit with
 * dot(d, ng) = cosg.  Returns 1 with out_dir and weight, or 0 when the path would end. */
ORC_API int orc_rough_scatter(const double *d, const double *ns, const double *ng, double n_lambda, double alpha,
                              double u0, double u1, double u2, int flags, double *out_dir, double *weight,
                              int *reflected) {
  surf f;
  memset(&f, 0, sizeof(f));
  v3 dv = V(d[0], d[1], d[2]);
  f.ng = V(ng[0], ng[1], ng[2]);
  f.ns = V(ns[0], ns[1], ns[2]);
  f.cosg = dot(dv, f.ng);
  double side = f.cosg < 0 ? 1.0 : -1.0;
  f.ngf = mul(f.ng, side);
  f.nsf = mul(f.ns, side);
  tolerances tol = DEFAULT_TOL;
  actx a;
  actx_init(&a, &tol);
  v3 o = V(0, 0, 0);
  int fix;
  int ok = rough_dielectric(&f, dv, n_lambda, alpha, u0, u1, u2, flags, &o, weight, reflected, &fix, &a);
  out_dir[0] = o.x; out_dir[1] = o.y; out_dir[2] = o.z;
  return ok;
}

/* Beer-Lambert attenuation of a segment of length t inside a dielectric */
static v3 absorb_over(const material *m, double t) {
  return V(exp(-m->absorb.x * t), exp(-m->absorb.y * t), exp(-m->absorb.z * t));
}

/* ------------------------------------------------------------------------------------------ */
/* parameters and records (layouts mirrored in oracle/__init__.py)                             */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  int32_t spp, sample_offset, max_depth, nbins;
  uint64_t seed;
  int32_t scene_index, flags;
  int32_t x0, x1, y0, y1; /* pixel window [x0,x1) x [y0,y1) */
  int32_t n_threads, brute;
  tolerances tol;
} cam_params;

typedef struct {
  double L[3];
  double p0[3];
  int32_t first_tri, n_queries;
  uint32_t signature;
  int32_t amb, bin, n_specular;
  double min_ratio;
  int32_t ratio_nspec, ratio_kind;
  double kmin[9];
  int32_t knspec[9], pad2;
} path_rec;

typedef struct {
  int64_t n_paths, path_offset;
  int32_t max_depth, nbins;
  uint64_t seed;
  int32_t scene_index, flags;
  int32_t n_threads, brute;
  tolerances tol;
  double guide[4]; /* sphere enclosing the dielectric triangles (centre, radius); radius <= 0: none */
} light_params;

typedef struct {
  double C[3];
  double x[3];
  int32_t pixel, amb;
  uint32_t signature;
  int32_t n_specular, bin, pad;
  double min_ratio;
  int32_t ratio_nspec, ratio_kind;
  double kmin[9];
  int32_t knspec[9], pad2;
  /* photon of the local-caustic estimate: deposited at the first diffuse vertex after at least
   * one specular event (photon = 1), with the path throughput there (no spectral weight) and the
   * shading normal on the side the light came from */
  double beta[3];
  double n[3];
  int32_t photon, pad3;
} light_rec;

static uint32_t fnv(uint32_t h, uint32_t w) { return (h ^ w) * 16777619u; }

/* pinhole ray through film position (sx, sy) in [0,1)^2, y down */
static ray camera_ray(const scene *s, double sx, double sy) {
  v3 d = add(add(mul(s->r, (2.0 * sx - 1.0) * s->th * s->aspect), mul(s->u, (1.0 - 2.0 * sy) * s->th)), s->f);
  ray r = {s->eye, normalize(d)};
  return r;
}

/* next-event estimate at a diffuse vertex (without the throughput) */
static v3 nee(const scene *s, const surf *f, v3 albedo, const uint32_t x[4], int brute, int *lit, actx *a) {
  const tolerances *tol = a->tol;
  *lit = 0;
  if (s->nlights == 0) return V(0, 0, 0);
  int j = choose(x[0], s->nlights);
  const light *L = &s->lights[j];
  v3 lp, le;
  double geo;
  if (L->kind == LIGHT_POINT) {
    lp = L->p; le = L->power;
    v3 w = sub(lp, f->p);
    double d2 = dot(w, w);
    w = mul(w, 1.0 / sqrt(d2));
    double cs = dot(f->nsf, w), cg = dot(f->ngf, w);
    note(a, fabs(cg), tol->cosg, AMB_GRAZE);
    note(a, fabs(cs), tol->cosg, 4);
    if (!(cs > 0 && cg > 0)) return V(0, 0, 0);
    geo = cs / d2;
  } else if (L->kind == LIGHT_RECT) {
    double ua = u01(x[1]), ub = u01(x[2]);
    lp = add(add(L->p, mul(L->u, ua)), mul(L->v, ub));
    le = L->power;
    v3 c = cross(L->u, L->v);
    double area = len(c);
    v3 nl = mul(c, 1.0 / area);
    v3 w = sub(lp, f->p);
    double d2 = dot(w, w);
    w = mul(w, 1.0 / sqrt(d2));
    double cs = dot(f->nsf, w), cg = dot(f->ngf, w), cl = -dot(nl, w);
    note(a, fabs(cg), tol->cosg, 4);
    note(a, fabs(cs), tol->cosg, 4);
    note(a, fabs(cl), tol->cosg, 4);
    if (!(cs > 0 && cg > 0 && cl > 0)) return V(0, 0, 0);
    geo = cs * cl * area / d2;
  } else {
    return V(0, 0, 0);
  }
  ray sr;
  sr.o = add(f->p, mul(f->ngf, eps_of(f->p)));
  v3 w = sub(lp, sr.o);
  double dist = len(w);
  sr.d = mul(w, 1.0 / dist);
  int occ = occluded_noted(s, sr, dist * (1.0 - 1e-4), brute, a);
  if (occ) return V(0, 0, 0);
  *lit = 1;
  return mul(hadamard(albedo, le), geo * (double)s->nlights / PI);
}

/* Sensitivity re-traces: the same path with its ray nudged after every scattering event by a
 * deterministic pseudo-random offset of relative size delta (a few float32 ulps or more).  A path
 * whose decisions or radiance move under such nudges cannot be reproduced by a float32 tracer
 * decision for decision, whatever its local margins. */
/* the re-traces: two perturbation directions (stream salts) times both signs */
static const uint64_t NUDGE_SALT[2] = {0xA5A5A5A5ull, 0x3C3C3C3C5A5A5A5Aull};
static void nudge(ray *r, double delta, uint64_t seed, uint32_t c0, uint32_t c1, int k) {
  if (delta == 0.0) return;
  uint32_t x[4], y[4];
  draw(seed, c0, c1, (uint32_t)k, 7, 0, x);
  draw(seed, c0, c1, (uint32_t)k, 8, 0, y);
  v3 a = V(2.0 * u01(x[0]) - 1.0, 2.0 * u01(x[1]) - 1.0, 2.0 * u01(x[2]) - 1.0);
  v3 b = V(2.0 * u01(y[0]) - 1.0, 2.0 * u01(y[1]) - 1.0, 2.0 * u01(y[2]) - 1.0);
  r->o = add(r->o, mul(a, delta * fmax(1.0, maxabs(r->o))));
  r->d = normalize(add(r->d, mul(b, delta)));
}

static int sensitive3(const double *a, const double *b, double rel) {
  for (int c = 0; c < 3; ++c) {
    double sc = fmax(fmax(fabs(a[c]), fabs(b[c])), 1e-6);
    if (fabs(a[c] - b[c]) > rel * sc) return 1;
  }
  return 0;
}

static void camera_path_impl(const scene *s, const cam_params *P, const double *wts, int px, int py,
                             int sample, double delta, uint64_t salt, path_rec *rec) {
  actx a;
  actx_init(&a, &P->tol);
  uint32_t pix = (uint32_t)(py * s->W + px);
  uint32_t x[4];
  draw(P->seed, pix, (uint32_t)sample, 0, 0, (uint32_t)P->scene_index, x);
  spec_sample sp = spectral_sample(x[2], P->nbins, P->flags, wts);
  int bin = sp.bin;
  ray r = camera_ray(s, (px + u01(x[0])) / s->W, (py + u01(x[1])) / s->H);
  nudge(&r, delta, P->seed ^ salt, pix, (uint32_t)sample, 0);
  v3 beta = V(1, 1, 1), L = V(0, 0, 0);
  int spec_only = 1, diffuse_first = 0, n_diffuse = 0, q = 0;
  uint32_t sig = 2166136261u;
  rec->first_tri = -1;
  rec->p0[0] = rec->p0[1] = rec->p0[2] = NAN;
  int last_specular = 0;
  for (int k = 0; k < P->max_depth; ++k) {
    hit h = closest_noted(s, r, P->brute, &a);
    ++q;
    sig = fnv(sig, h.tri < 0 ? EV_MISS : (uint32_t)h.tri);
    if (k == 0) rec->first_tri = h.tri;
    if (h.tri < 0) { L = add(L, hadamard(beta, s->env)); break; }
    surf f = interact(s, r, h);
    if (k == 0) { rec->p0[0] = f.p.x; rec->p0[1] = f.p.y; rec->p0[2] = f.p.z; }
    note(&a, fabs(f.cosg), P->tol.cosg, AMB_GRAZE);
    const material *m = &s->mats[f.mat];
    /* a segment that ends on a dielectric's inner side ran through that glass */
    if (m->kind == MAT_DIELECTRIC && f.cosg > 0) beta = hadamard(beta, absorb_over(m, h.t));
    if (m->kind == MAT_EMISSIVE) {
      int count = spec_only || ((P->flags & FLAG_EMITTER_AFTER_DS) && diffuse_first && n_diffuse == 1 &&
                                last_specular);
      if (f.cosg < 0 && count) L = add(L, hadamard(beta, m->emission));
      break;
    }
    uint32_t xs[4];
    draw(P->seed, pix, (uint32_t)sample, (uint32_t)(k + 1), 1, (uint32_t)P->scene_index, xs);
    if (m->kind == MAT_DIELECTRIC) {
      int refl, fix;
      double n_l = cauchy_at(m->A, m->B, sp.lam, P->nbins);
      v3 d;
      if (m->alpha > 0) {
        double wgt;
        int ok = rough_dielectric(&f, r.d, n_l, m->alpha, u01(xs[0]), u01(xs[1]), u01(xs[2]), P->flags, &d, &wgt,
                                  &refl, &fix, &a);
        if (!ok) { sig = fnv(sig, EV_KILL); ++a.nspec; break; }
        beta = mul(beta, wgt);
      } else {
        d = dielectric(&f, r.d, n_l, u01(xs[0]), P->flags, &refl, &fix, &a);
      }
      sig = fnv(sig, refl ? EV_REFLECT : EV_REFRACT);
      if (fix) sig = fnv(sig, EV_FIXUP);
      ++a.nspec;
      last_specular = 1;
      r.o = offset_along(f.p, f.ng, d);
      r.d = d;
      nudge(&r, delta, P->seed ^ salt, pix, (uint32_t)sample, k + 1);
      continue;
    }
    /* diffuse */
    v3 alb = albedo_at(s, h.tri, &f, &a);
    uint32_t xn[4];
    draw(P->seed, pix, (uint32_t)sample, (uint32_t)(k + 1), 2, (uint32_t)P->scene_index, xn);
    int lit;
    v3 e = nee(s, &f, alb, xn, P->brute, &lit, &a);
    sig = fnv(sig, lit ? EV_LIT : EV_UNLIT);
    L = add(L, hadamard(beta, e));
    if (k == 0) diffuse_first = 1;
    ++n_diffuse;
    spec_only = 0;
    last_specular = 0;
    if (k == P->max_depth - 1) break;
    v3 d = cosine_dir(f.nsf, u01(xs[1]), u01(xs[2]));
    double side = dot(d, f.ngf);
    note(&a, fabs(side), P->tol.cosg, AMB_FIXUP);
    if (!(side > 0)) {
      d = cosine_dir(f.ngf, u01(xs[1]), u01(xs[2]));
      sig = fnv(sig, EV_FIXUP);
    }
    beta = hadamard(beta, alb);
    r.o = add(f.p, mul(f.ngf, eps_of(f.p)));
    r.d = d;
    nudge(&r, delta, P->seed ^ salt, pix, (uint32_t)sample, k + 1);
  }
  L = hadamard(L, sp.w);
  rec->L[0] = L.x; rec->L[1] = L.y; rec->L[2] = L.z;
  rec->n_queries = q;
  rec->signature = sig;
  rec->amb = a.amb;
  rec->bin = bin;
  rec->n_specular = a.nspec;
  rec->min_ratio = a.min_ratio;
  rec->ratio_nspec = a.ratio_nspec;
  rec->ratio_kind = a.ratio_kind;
  for (int i = 0; i < 9; ++i) { rec->kmin[i] = a.kmin[i]; rec->knspec[i] = a.knspec[i]; }
}

static void camera_path(const scene *s, const cam_params *P, const double *wts, int px, int py, int sample,
                        path_rec *rec) {
  camera_path_impl(s, P, wts, px, py, sample, 0.0, 0, rec);
  if (P->tol.sens_delta > 0) {
    for (int v = 0; v < 2 && !(rec->amb & AMB_SENSITIVE); ++v)
      for (int sgn = -1; sgn <= 1; sgn += 2) {
        path_rec alt;
        camera_path_impl(s, P, wts, px, py, sample, sgn * P->tol.sens_delta, NUDGE_SALT[v], &alt);
        if (alt.signature != rec->signature || sensitive3(alt.L, rec->L, P->tol.sens_rel)) rec->amb |= AMB_SENSITIVE;
      }
  }
}

/* Local caustics (caustics seen through glass, E S+ D S+ L; Sec. III-D "Local & Non-local
 * Caustics Mask"): a camera path's prefix, traced exactly as the camera estimator traces it (same
 * draws, same dielectric events), up to its first non-dielectric hit.  If that is a diffuse
 * surface reached after at least one dielectric event, the path gathers photons there; the
 * record holds the gather point, its shading normal on the camera's side, the bin, and the
 * camera-side weight w = beta * albedo / pi * W(lambda) (RGB).  Photon density estimation itself
 * (photons of the same bin within the radius, normals on the same side) is done by the caller. */
typedef struct {
  double x[3], n[3], w[3];
  int32_t valid, bin, amb, n_specular;
  uint32_t signature, pad;
} gather_rec;

static void gather_path(const scene *s, const cam_params *P, const double *wts, int px, int py, int sample,
                        gather_rec *rec) {
  actx a;
  actx_init(&a, &P->tol);
  memset(rec, 0, sizeof(*rec));
  uint32_t pix = (uint32_t)(py * s->W + px);
  uint32_t x[4];
  draw(P->seed, pix, (uint32_t)sample, 0, 0, (uint32_t)P->scene_index, x);
  spec_sample sp = spectral_sample(x[2], P->nbins, P->flags, wts);
  rec->bin = sp.bin;
  ray r = camera_ray(s, (px + u01(x[0])) / s->W, (py + u01(x[1])) / s->H);
  v3 beta = V(1, 1, 1);
  uint32_t sig = 2166136261u;
  for (int k = 0; k < P->max_depth; ++k) {
    hit h = closest_noted(s, r, P->brute, &a);
    sig = fnv(sig, h.tri < 0 ? EV_MISS : (uint32_t)h.tri);
    if (h.tri < 0) break;
    surf f = interact(s, r, h);
    note(&a, fabs(f.cosg), P->tol.cosg, AMB_GRAZE);
    const material *m = &s->mats[f.mat];
    if (m->kind == MAT_DIELECTRIC && f.cosg > 0) beta = hadamard(beta, absorb_over(m, h.t));
    if (m->kind == MAT_EMISSIVE) break;
    if (m->kind == MAT_DIELECTRIC) {
      uint32_t xs[4];
      draw(P->seed, pix, (uint32_t)sample, (uint32_t)(k + 1), 1, (uint32_t)P->scene_index, xs);
      int refl, fix;
      double n_l = cauchy_at(m->A, m->B, sp.lam, P->nbins);
      v3 d;
      if (m->alpha > 0) {
        double wgt;
        int ok = rough_dielectric(&f, r.d, n_l, m->alpha, u01(xs[0]), u01(xs[1]), u01(xs[2]), P->flags, &d, &wgt,
                                  &refl, &fix, &a);
        if (!ok) { sig = fnv(sig, EV_KILL); ++a.nspec; break; }
        beta = mul(beta, wgt);
      } else {
        d = dielectric(&f, r.d, n_l, u01(xs[0]), P->flags, &refl, &fix, &a);
      }
      sig = fnv(sig, refl ? EV_REFLECT : EV_REFRACT);
      if (fix) sig = fnv(sig, EV_FIXUP);
      ++a.nspec;
      r.o = offset_along(f.p, f.ng, d);
      r.d = d;
      continue;
    }
    /* diffuse: the gather vertex when reached through glass */
    if (a.nspec > 0) {
      v3 alb = albedo_at(s, h.tri, &f, &a);
      v3 w = hadamard(hadamard(beta, alb), sp.w);
      rec->valid = 1;
      rec->x[0] = f.p.x; rec->x[1] = f.p.y; rec->x[2] = f.p.z;
      rec->n[0] = f.nsf.x; rec->n[1] = f.nsf.y; rec->n[2] = f.nsf.z;
      rec->w[0] = w.x / PI; rec->w[1] = w.y / PI; rec->w[2] = w.z / PI;
    }
    break;
  }
  rec->amb = a.amb;
  rec->n_specular = a.nspec;
  rec->signature = sig;
}

/* one gather record per (pixel, sample) of the window, row-major, samples innermost */
ORC_API void orc_trace_gather(void *sp, const cam_params *P, gather_rec *recs) {
  const scene *s = sp;
  double *wts = malloc(sizeof(double) * 3 * (size_t)(P->nbins > 1 ? P->nbins : 1));
  orc_spectral_weights(P->nbins, wts, NULL);
  int64_t i = 0;
  for (int py = P->y0; py < P->y1; ++py)
    for (int px = P->x0; px < P->x1; ++px)
      for (int smp = 0; smp < P->spp; ++smp) gather_path(s, P, wts, px, py, P->sample_offset + smp, &recs[i++]);
  free(wts);
}

/* ------------------------------------------------------------------------------------------ */
/* light path (caustics)                                                                       */
/* ------------------------------------------------------------------------------------------ */

/* Guided emission: a direction uniform in the cone that subtends the guide sphere (centre g[0..2],
 * radius g[3]) from x, drawn from (u0, u1) as cos(theta) = 1 - u0 (1 - cos(theta_max)),
 * phi = 2 pi u1 about the axis x -> centre.  Returns the cone's solid angle 2 pi (1 - cos
 * theta_max), or 0 (no direction drawn) when there is no guide or x lies inside the sphere. */
static double guided_dir(const double *g, v3 x, double u0, double u1, v3 *dir) {
  if (!(g[3] > 0)) return 0.0;
  v3 v = sub(V(g[0], g[1], g[2]), x);
  double dist = len(v);
  if (!(dist > g[3])) return 0.0;
  v3 w = mul(v, 1.0 / dist), t1, t2;
  double sin2 = (g[3] / dist) * (g[3] / dist);
  double cmax = sqrt(fmax(0.0, 1.0 - sin2));
  double omc = sin2 / (1.0 + cmax); /* 1 - cos(theta_max) */
  double ct = 1.0 - u0 * omc, st = sqrt(fmax(0.0, 1.0 - ct * ct)), phi = 2.0 * PI * u1;
  onb(w, &t1, &t2);
  *dir = normalize(add(add(mul(t1, st * cos(phi)), mul(t2, st * sin(phi))), mul(w, ct)));
  return 2.0 * PI * omc;
}
static void light_path_impl(const scene *s, const light_params *P, const double *wts, int64_t idx, double delta,
                            uint64_t salt,
                            double *accum, light_rec *rec) {
  actx a;
  actx_init(&a, &P->tol);
  uint32_t lo = (uint32_t)idx, hi = (uint32_t)((uint64_t)idx >> 32);
  uint32_t xe[4], xd[4];
  draw(P->seed, lo, hi, 0, 4, (uint32_t)P->scene_index, xe);
  draw(P->seed, lo, hi, 0, 3, (uint32_t)P->scene_index, xd);
  spec_sample sp = spectral_sample(xe[3], P->nbins, P->flags, wts);
  int bin = sp.bin;
  uint32_t sig = 2166136261u;
  rec->pixel = -1;
  rec->C[0] = rec->C[1] = rec->C[2] = 0;
  rec->x[0] = rec->x[1] = rec->x[2] = NAN;
  rec->bin = bin;
  rec->photon = 0;
  rec->beta[0] = rec->beta[1] = rec->beta[2] = 0;
  rec->n[0] = rec->n[1] = rec->n[2] = 0;
  if (s->nlights == 0) goto done;
  {
    int j = choose(xe[0], s->nlights);
    const light *L = &s->lights[j];
    ray r;
    v3 beta;
    int emitted = 1;
    if (L->kind == LIGHT_POINT) {
      double z = 1.0 - 2.0 * u01(xd[0]), phi = 2.0 * PI * u01(xd[1]);
      double rr = sqrt(fmax(0.0, 1.0 - z * z));
      r.o = L->p;
      double omega = guided_dir(P->guide, r.o, u01(xd[0]), u01(xd[1]), &r.d);
      if (omega > 0) {
        beta = mul(L->power, omega * s->nlights);
      } else {
        r.d = normalize(V(rr * cos(phi), rr * sin(phi), z));
        beta = mul(L->power, 4.0 * PI * s->nlights);
      }
    } else if (L->kind == LIGHT_RECT) {
      v3 c = cross(L->u, L->v);
      double area = len(c);
      v3 nl = mul(c, 1.0 / area);
      v3 x = add(add(L->p, mul(L->u, u01(xe[1]))), mul(L->v, u01(xe[2])));
      double omega = guided_dir(P->guide, x, u01(xd[0]), u01(xd[1]), &r.d);
      if (omega > 0) {
        double cl = dot(r.d, nl);
        note(&a, fabs(cl), P->tol.cosg, AMB_GRAZE);
        emitted = cl > 0; /* one-sided emitter */
        beta = mul(L->power, area * s->nlights * cl * omega);
      } else {
        r.d = cosine_dir(nl, u01(xd[0]), u01(xd[1]));
        beta = mul(L->power, PI * area * s->nlights);
      }
      r.o = add(x, mul(nl, eps_of(x)));
    } else {
      v3 dir = normalize(L->u), t1, t2;
      onb(dir, &t1, &t2);
      double rad = L->radius * sqrt(u01(xe[1])), phi = 2.0 * PI * u01(xe[2]);
      r.o = add(L->p, add(mul(t1, rad * cos(phi)), mul(t2, rad * sin(phi))));
      r.d = dir;
      beta = mul(L->power, PI * L->radius * L->radius * s->nlights);
    }
    int had_spec = 0;
    nudge(&r, delta, P->seed ^ salt, lo, hi, 0);
    for (int k = 0; emitted && k < P->max_depth; ++k) {
      hit h = closest_noted(s, r, P->brute, &a);
      sig = fnv(sig, h.tri < 0 ? EV_MISS : (uint32_t)h.tri);
      if (h.tri < 0) break;
      surf f = interact(s, r, h);
      note(&a, fabs(f.cosg), P->tol.cosg, AMB_GRAZE);
      const material *m = &s->mats[f.mat];
      if (m->kind == MAT_DIELECTRIC && f.cosg > 0) beta = hadamard(beta, absorb_over(m, h.t));
      if (m->kind == MAT_EMISSIVE) break;
      if (m->kind == MAT_DIELECTRIC) {
        uint32_t xs[4];
        draw(P->seed, lo, hi, (uint32_t)(k + 1), 3, (uint32_t)P->scene_index, xs);
        int refl, fix;
        double n_l = cauchy_at(m->A, m->B, sp.lam, P->nbins);
        v3 d;
        if (m->alpha > 0) {
          double wgt;
          int ok = rough_dielectric(&f, r.d, n_l, m->alpha, u01(xs[0]), u01(xs[1]), u01(xs[2]), P->flags, &d,
                                    &wgt, &refl, &fix, &a);
          if (!ok) { sig = fnv(sig, EV_KILL); ++a.nspec; break; }
          beta = mul(beta, wgt);
        } else {
          d = dielectric(&f, r.d, n_l, u01(xs[0]), P->flags, &refl, &fix, &a);
        }
        sig = fnv(sig, refl ? EV_REFLECT : EV_REFRACT);
        if (fix) sig = fnv(sig, EV_FIXUP);
        ++a.nspec;
        had_spec = 1;
        r.o = offset_along(f.p, f.ng, d);
        r.d = d;
        nudge(&r, delta, P->seed ^ salt, lo, hi, k + 1);
        continue;
      }
      /* diffuse receiver */
      if (!had_spec && !(P->flags & FLAG_SPLAT_DIRECT)) break;
      rec->x[0] = f.p.x; rec->x[1] = f.p.y; rec->x[2] = f.p.z;
      if (had_spec) {
        rec->photon = 1;
        rec->beta[0] = beta.x; rec->beta[1] = beta.y; rec->beta[2] = beta.z;
        rec->n[0] = f.nsf.x; rec->n[1] = f.nsf.y; rec->n[2] = f.nsf.z;
      }
      v3 alb = albedo_at(s, h.tri, &f, &a);
      v3 wc = sub(s->eye, f.p);
      double dc = len(wc);
      wc = mul(wc, 1.0 / dc);
      double cs = dot(f.nsf, wc), cg = dot(f.ngf, wc);
      note(&a, fabs(cg), P->tol.cosg, 4);
      note(&a, fabs(cs), P->tol.cosg, 4);
      if (!(cs > 0 && cg > 0)) { sig = fnv(sig, EV_UNLIT); break; }
      v3 wv = mul(wc, -1.0);
      double cc = dot(wv, s->f);
      if (!(cc > 0)) { sig = fnv(sig, EV_UNLIT); break; }
      double sx = (dot(wv, s->r) / cc / (s->th * s->aspect) + 1.0) * 0.5;
      double sy = (1.0 - dot(wv, s->u) / cc / s->th) * 0.5;
      double fx = sx * s->W, fy = sy * s->H;
      note(&a, fmin(fabs(fx - floor(fx + 0.5)), fabs(fy - floor(fy + 0.5))), P->tol.px, AMB_SPLAT);
      if (!(sx >= 0 && sx < 1 && sy >= 0 && sy < 1)) { sig = fnv(sig, EV_UNLIT); break; }
      int ix = (int)floor(fx), iy = (int)floor(fy);
      if (ix >= s->W) ix = s->W - 1;
      if (iy >= s->H) iy = s->H - 1;
      ray sr;
      sr.o = add(f.p, mul(f.ngf, eps_of(f.p)));
      v3 w = sub(s->eye, sr.o);
      double dist = len(w);
      sr.d = mul(w, 1.0 / dist);
      int occ = occluded_noted(s, sr, dist * (1.0 - 1e-4), P->brute, &a);
      if (occ) { sig = fnv(sig, EV_UNLIT); break; }
      sig = fnv(sig, EV_LIT);
      double apix = (2.0 * s->th * s->aspect / s->W) * (2.0 * s->th / s->H);
      double g = cs / (dc * dc * apix * cc * cc * cc) / PI;
      v3 C = hadamard(hadamard(mul(beta, g), alb), sp.w);
      rec->pixel = iy * s->W + ix;
      rec->C[0] = C.x; rec->C[1] = C.y; rec->C[2] = C.z;
      if (accum) {
        double *a3 = accum + 3 * (size_t)rec->pixel;
        a3[0] += C.x; a3[1] += C.y; a3[2] += C.z;
      }
      break;
    }
  }
done:
  rec->amb = a.amb;
  rec->signature = sig;
  rec->n_specular = a.nspec;
  rec->min_ratio = a.min_ratio;
  rec->ratio_nspec = a.ratio_nspec;
  rec->ratio_kind = a.ratio_kind;
  for (int i = 0; i < 9; ++i) { rec->kmin[i] = a.kmin[i]; rec->knspec[i] = a.knspec[i]; }
}

static void light_path(const scene *s, const light_params *P, const double *wts, int64_t idx, double *accum,
                       light_rec *rec) {
  light_path_impl(s, P, wts, idx, 0.0, 0, accum, rec);
  if (P->tol.sens_delta > 0) {
    for (int v = 0; v < 2 && !(rec->amb & AMB_SENSITIVE); ++v)
      for (int sgn = -1; sgn <= 1; sgn += 2) {
        light_rec alt;
        light_path_impl(s, P, wts, idx, sgn * P->tol.sens_delta, NUDGE_SALT[v] ^ 0xFFull, NULL, &alt);
        if (alt.signature != rec->signature || alt.pixel != rec->pixel || sensitive3(alt.C, rec->C, P->tol.sens_rel))
          rec->amb |= AMB_SENSITIVE;
      }
  }
}

/* ------------------------------------------------------------------------------------------ */
/* threaded drivers                                                                            */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  const scene *s;
  const cam_params *cp;
  const light_params *lp;
  const double *wts;
  double *accum;
  path_rec *crec;
  light_rec *lrec;
  int64_t next, total, chunk;
  double *scratch; /* per-thread light accumulators */
  int nthreads;
  pthread_mutex_t lock;
} job;

static void *cam_worker(void *arg) {
  job *J = arg;
  const cam_params *P = J->cp;
  int ww = P->x1 - P->x0;
  for (;;) {
    int64_t row = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
    if (row >= J->total) break;
    int py = P->y0 + (int)row;
    for (int px = P->x0; px < P->x1; ++px) {
      double acc[3] = {0, 0, 0};
      for (int sidx = 0; sidx < P->spp; ++sidx) {
        path_rec rec;
        camera_path(J->s, P, J->wts, px, py, P->sample_offset + sidx, &rec);
        acc[0] += rec.L[0]; acc[1] += rec.L[1]; acc[2] += rec.L[2];
        if (J->crec) J->crec[((int64_t)row * ww + (px - P->x0)) * P->spp + sidx] = rec;
      }
      if (J->accum) {
        double *a = J->accum + 3 * ((int64_t)py * J->s->W + px);
        a[0] += acc[0]; a[1] += acc[1]; a[2] += acc[2];
      }
    }
  }
  return NULL;
}

static int thread_count(int req) {
  if (req > 0) return req;
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  return n > 0 ? (int)n : 1;
}

/* Adds the camera estimator's radiance sums for the window into accum (W*H*3, may be NULL) and
 * writes one record per path (window rows x window cols x spp, may be NULL). */
ORC_API int orc_trace_camera(void *sp, const cam_params *P, double *accum, path_rec *recs) {
  const scene *s = sp;
  double *wts = malloc(sizeof(double) * 3 * (size_t)(P->nbins > 1 ? P->nbins : 1));
  orc_spectral_weights(P->nbins, wts, NULL);
  job J;
  memset(&J, 0, sizeof(J));
  J.s = s; J.cp = P; J.wts = wts; J.accum = accum; J.crec = recs;
  J.next = 0; J.total = P->y1 - P->y0;
  int nt = thread_count(P->n_threads);
  pthread_t th[256];
  if (nt > 256) nt = 256;
  for (int i = 0; i < nt; ++i) pthread_create(&th[i], NULL, cam_worker, &J);
  for (int i = 0; i < nt; ++i) pthread_join(th[i], NULL);
  free(wts);
  return nt;
}

static void *light_worker(void *arg) {
  job *J = arg;
  const light_params *P = J->lp;
  size_t npix = (size_t)J->s->W * J->s->H;
  int tid;
  pthread_mutex_lock(&J->lock);
  tid = J->nthreads++;
  pthread_mutex_unlock(&J->lock);
  double *acc = J->scratch ? J->scratch + 3 * npix * (size_t)tid : NULL;
  for (;;) {
    int64_t c = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
    int64_t a = c * J->chunk;
    if (a >= J->total) break;
    int64_t b = a + J->chunk < J->total ? a + J->chunk : J->total;
    for (int64_t i = a; i < b; ++i) {
      light_rec rec;
      light_path(J->s, P, J->wts, P->path_offset + i, acc, &rec);
      if (J->lrec) J->lrec[i] = rec;
    }
  }
  return NULL;
}

/* Adds the raw (not yet divided by the path count) splat sums into accum (W*H*3, may be NULL)
 * and writes one record per light path (may be NULL). */
ORC_API int orc_trace_lights(void *sp, const light_params *P, double *accum, light_rec *recs) {
  const scene *s = sp;
  double *wts = malloc(sizeof(double) * 3 * (size_t)(P->nbins > 1 ? P->nbins : 1));
  orc_spectral_weights(P->nbins, wts, NULL);
  int nt = thread_count(P->n_threads);
  if (nt > 256) nt = 256;
  size_t npix = (size_t)s->W * s->H;
  job J;
  memset(&J, 0, sizeof(J));
  J.s = s; J.lp = P; J.wts = wts; J.lrec = recs;
  J.next = 0; J.total = P->n_paths; J.chunk = 4096;
  pthread_mutex_init(&J.lock, NULL);
  J.scratch = accum ? calloc(3 * npix * (size_t)nt, sizeof(double)) : NULL;
  pthread_t th[256];
  for (int i = 0; i < nt; ++i) pthread_create(&th[i], NULL, light_worker, &J);
  for (int i = 0; i < nt; ++i) pthread_join(th[i], NULL);
  if (accum) {
    for (int t = 0; t < nt; ++t)
      for (size_t i = 0; i < 3 * npix; ++i) accum[i] += J.scratch[3 * npix * (size_t)t + i];
    free(J.scratch);
  }
  pthread_mutex_destroy(&J.lock);
  free(wts);
  return nt;
}

/* ------------------------------------------------------------------------------------------ */
/* resolve and ground-truth buffers (pixel-centre primary ray, no random numbers)              */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  double spp_total, light_paths_total, depth_range, tau_rel;
  int32_t brute, pad;
} resolve_params;

typedef struct {
  double rgb[3], direct[3], caustic[3];
  double depth, depth_norm;
  double n_world[3], n_cam[3], albedo[3];
  int32_t instance, tri, mask, caustic_mask, local_caustic_mask, amb;
  double local_caustic[3];
} pixel_out;

static double luminance(const double *c) { return 0.2126 * c[0] + 0.7152 * c[1] + 0.0722 * c[2]; }

/* acc_local (may be NULL): sums over the spp_total camera samples of the local-caustic gather */
ORC_API void orc_resolve(void *sp, const resolve_params *P, const double *acc_cam, const double *acc_caus,
                         const double *acc_local, pixel_out *out) {
  const scene *s = sp;
  for (int py = 0; py < s->H; ++py)
    for (int px = 0; px < s->W; ++px) {
      int64_t i = (int64_t)py * s->W + px;
      pixel_out *o = &out[i];
      memset(o, 0, sizeof(*o));
      for (int c = 0; c < 3; ++c) {
        o->direct[c] = acc_cam ? acc_cam[3 * i + c] / P->spp_total : 0.0;
        o->caustic[c] = (acc_caus && P->light_paths_total > 0) ? acc_caus[3 * i + c] / P->light_paths_total : 0.0;
        o->local_caustic[c] = (acc_local && P->spp_total > 0) ? acc_local[3 * i + c] / P->spp_total : 0.0;
        o->rgb[c] = o->direct[c] + o->caustic[c] + o->local_caustic[c];
      }
      actx a;
      actx_init(&a, &DEFAULT_TOL);
      ray r = camera_ray(s, (px + 0.5) / s->W, (py + 0.5) / s->H);
      hit h = closest_noted(s, r, P->brute, &a);
      if (h.tri < 0) {
        o->instance = -1; o->tri = -1; o->depth = INFINITY; o->depth_norm = 1.0; o->amb = a.amb;
        continue;
      }
      surf f = interact(s, r, h);
      note(&a, fabs(f.cosg), DEFAULT_TOL.cosg, 4);
      const material *m = &s->mats[f.mat];
      o->instance = s->obj[h.tri];
      o->tri = h.tri;
      o->mask = m->kind == MAT_DIELECTRIC;
      o->depth = len(sub(f.p, s->eye));
      o->depth_norm = fmin(o->depth / P->depth_range, 1.0);
      v3 n = f.nsf;
      o->n_world[0] = n.x; o->n_world[1] = n.y; o->n_world[2] = n.z;
      o->n_cam[0] = dot(n, s->r); o->n_cam[1] = dot(n, s->u); o->n_cam[2] = -dot(n, s->f);
      v3 alb = m->kind == MAT_DIFFUSE ? albedo_at(s, h.tri, &f, &a) : V(1, 1, 1);
      o->amb = a.amb;
      o->albedo[0] = alb.x; o->albedo[1] = alb.y; o->albedo[2] = alb.z;
      double yc = luminance(o->caustic), yd = luminance(o->direct);
      o->caustic_mask = (m->kind != MAT_DIELECTRIC) && (yc > P->tau_rel * fmax(yd, 1e-3));
      /* local caustics: seen through the glass of this pixel (the with / without difference is the
       * local-caustic buffer) */
      o->local_caustic_mask = (m->kind == MAT_DIELECTRIC) && (luminance(o->local_caustic) > P->tau_rel * fmax(yd, 1e-3));
    }
}

ORC_API int orc_sizes(int *out) {
  out[0] = (int)sizeof(cam_params);
  out[1] = (int)sizeof(path_rec);
  out[2] = (int)sizeof(light_params);
  out[3] = (int)sizeof(light_rec);
  out[4] = (int)sizeof(resolve_params);
  out[5] = (int)sizeof(pixel_out);
  out[6] = (int)sizeof(tolerances);
  out[7] = (int)sizeof(gather_rec);
  return 8;
}
