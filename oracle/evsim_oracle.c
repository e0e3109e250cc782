/*
 * Plain CPU oracle for the flow-interpolation event simulator.
 * TEST INFRASTRUCTURE ONLY: see evsim_oracle.h.  Every step is written in the
 * order the method defines it: substep-major, then rows, then columns, then
 * repeated crossings.  No blocking, no fusion, no SIMD, no threads.
 *
 * Paper: Ziegler et al., "Real-time event simulation with frame-based
 * cameras" (arXiv 2209.04634), Sec. III, III-A, III-B, III-C, Table I.
 */
#include "evsim_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* floor(a / b) for b > 0, rounding toward minus infinity. */
static int64_t floordiv(int64_t a, int64_t b) {
  int64_t q = a / b;
  if ((a % b != 0) && (a < 0)) q -= 1;
  return q;
}

/*
 * Intensity table.  Sec. III states the paper differences linear intensity;
 * the log reading takes the event-camera model of Sec. I (log-scale changes).
 *   ORC_LOG   : LUT[v] = round-half-even(65536 * ln(v + 1)); the +1 keeps
 *               v = 0 finite (the paper is silent on it).
 *   ORC_LINEAR: LUT[v] = v * 65536, thresholds then in 8-bit units as in
 *               Table I (C_pos = 2 / 10 / 20).
 */
void orc_lut(int32_t intensity, int32_t lut[256]) {
  for (int v = 0; v < 256; ++v) {
    if (intensity == ORC_LINEAR) {
      lut[v] = v * 65536;
    } else {
      double exact = 65536.0 * log((double)v + 1.0);
      lut[v] = (int32_t)nearbyint(exact); /* default rounding: ties to even */
    }
  }
}

/* BT.601 integer luma (the paper's inputs are grey-scale frames, Fig. 5a). */
int32_t orc_luma(int32_t r, int32_t g, int32_t b) {
  return (77 * r + 150 * g + 29 * b + 128) >> 8;
}

/* Flow to Q16: NaN -> 0; clamp to +-1024 px; nearest, ties to even.
 * *clamped is incremented once per clamped component. */
int32_t orc_flow_q16(float f, int32_t* clamped) {
  double d = (double)f;
  if (d != d) return 0;
  if (d > 1024.0) { d = 1024.0; if (clamped) *clamped += 1; }
  if (d < -1024.0) { d = -1024.0; if (clamped) *clamped += 1; }
  return (int32_t)nearbyint(d * 65536.0);
}

/* Linear blend of two Q16 values with a Q12 weight w in [0, 4096]:
 * a + floor(((b - a) * w + 2048) / 4096), i.e. round half up. */
static int64_t lerp_q12(int64_t a, int64_t b, int64_t w) {
  return a + floordiv((b - a) * w + 2048, 4096);
}

/*
 * Bilinear sample of a Q16 image at a Q16 position, the sampling step of the
 * "simple but fast linear interpolation" along the flow (Sec. III, III-A).
 * Borders (the paper is silent): the position is clamped to the image.
 * The fraction is the top 12 of the 16 fractional bits.
 */
int32_t orc_bilinear(const int32_t* L, int32_t W, int32_t H, int64_t px, int64_t py) {
  int64_t maxx = (int64_t)(W - 1) * 65536, maxy = (int64_t)(H - 1) * 65536;
  if (px < 0) px = 0;
  if (px > maxx) px = maxx;
  if (py < 0) py = 0;
  if (py > maxy) py = maxy;
  int64_t ix = px >> 16, iy = py >> 16;
  int64_t fx = (px & 0xFFFF) >> 4, fy = (py & 0xFFFF) >> 4;
  int64_t x1 = ix + 1 < W ? ix + 1 : W - 1;
  int64_t y1 = iy + 1 < H ? iy + 1 : H - 1;
  int64_t l00 = L[iy * W + ix], l01 = L[iy * W + x1];
  int64_t l10 = L[y1 * W + ix], l11 = L[y1 * W + x1];
  int64_t top = lerp_q12(l00, l01, fx);
  int64_t bot = lerp_q12(l10, l11, fx);
  return (int32_t)lerp_q12(top, bot, fy);
}

/* Smallest N >= 1 with N^2 * 2^32 >= max(Fx^2 + Fy^2), i.e. N = ceil(max|F|)
 * in pixels, capped at max_substeps.  The paper fixes N per data set
 * (Table I: 10; Sec. IV-A: 20 for the driving sequence); this is the
 * configuration's adaptive reading. */
int32_t orc_adaptive_substeps(int64_t max_f2, int32_t max_substeps) {
  int32_t n = 1;
  while (n < max_substeps && (int64_t)n * n * 4294967296LL < max_f2) ++n;
  return n;
}

/*
 * Per-crossing event time (reading O16; the paper's events carry a time t,
 * Sec. III, without saying where inside an interpolation step it falls).
 * Between two consecutive interpolated frames the pixel's value is taken to
 * change linearly in time, from i_prev at t_prev to i_cur at t_cur; a
 * threshold level crossed in that step is reached at
 *   t_prev + floor((t_cur - t_prev) (level - i_prev) / (i_cur - i_prev))
 * (mirrored for a falling value).  The levels an accumulating reference
 * crosses lie beyond i_prev and at or before i_cur, so the time falls in
 * (t_prev, t_cur]; a level at or behind i_prev (a sparse pixel whose
 * reference was left behind while it was inactive) gets t_prev.
 */
int64_t orc_crossing_time(int64_t t_prev, int64_t t_cur, int64_t i_prev, int64_t i_cur,
                          int64_t level, int32_t rising) {
  int64_t num = rising ? level - i_prev : i_prev - level;
  int64_t den = rising ? i_cur - i_prev : i_prev - i_cur;
  if (num <= 0 || den <= 0) return t_prev;
  return t_prev + floordiv((t_cur - t_prev) * num, den);
}

static int32_t pixel_threshold(const uint16_t* map, int32_t uniform, int64_t i) {
  return map ? (int32_t)map[i] : uniform;
}

static void emit(orc_event* out, int64_t cap, int64_t* n, uint32_t t, int32_t x,
                 int32_t y, int32_t pos) {
  if (*n < cap) {
    out[*n].t = t;
    out[*n].x = (uint16_t)x;
    out[*n].yp = (uint16_t)((y << 1) | (pos ? 1 : 0));
  }
  *n += 1;
}

static void frame_to_log(const orc_config* c, const int32_t lut[256], const uint8_t* f,
                         int32_t* L) {
  int64_t P = (int64_t)c->width * c->height;
  for (int64_t i = 0; i < P; ++i) {
    int32_t v;
    if (c->channels == 3)
      v = orc_luma(f[3 * i], f[3 * i + 1], f[3 * i + 2]);
    else
      v = f[i];
    L[i] = lut[v];
  }
}

int64_t orc_run(const orc_config* c, int32_t n_frames, const uint8_t* frames,
                const float* flows, const int64_t* t_us,
                const uint16_t* cpos_map, const uint16_t* cneg_map,
                orc_event* out, int64_t cap, int32_t* R_final,
                int32_t* n_per_frame, int64_t* ev_per_frame,
                int64_t* active_per_frame, int64_t* clamped_total) {
  if (!c || n_frames < 1 || !frames || !t_us || c->width < 1 || c->height < 1) return -1;
  if (c->channels != 1 && c->channels != 3) return -1;
  if (c->substeps < 0 || (c->substeps == 0 && c->max_substeps < 1)) return -1;
  if (n_frames > 1 && !flows) return -1;
  const int32_t W = c->width, H = c->height;
  const int64_t P = (int64_t)W * H;
  const int64_t fbytes = P * c->channels;
  /* the simulated rows [y0, y1) (a row band of a parallel run, or all rows) */
  const int32_t y0 = c->row_begin < 0 ? 0 : (c->row_begin > H ? H : c->row_begin);
  const int32_t y1 = c->row_end <= 0 || c->row_end > H ? H : c->row_end;
  const int64_t p_begin = (int64_t)y0 * W, p_end = (int64_t)(y1 > y0 ? y1 : y0) * W;
  /* the adaptive N is a maximum over the whole frame: then the flow and the
   * activity of every pixel are needed, else only those of the band */
  const int64_t q_begin = c->substeps == 0 ? 0 : p_begin;
  const int64_t q_end = c->substeps == 0 ? P : p_end;

  int32_t lut[256];
  orc_lut(c->intensity, lut);

  int32_t* Lprev = (int32_t*)malloc(P * sizeof(int32_t));
  int32_t* Lcur = (int32_t*)malloc(P * sizeof(int32_t));
  int32_t* R = (int32_t*)malloc(P * sizeof(int32_t));
  int32_t* Fx = (int32_t*)malloc(P * sizeof(int32_t));
  int32_t* Fy = (int32_t*)malloc(P * sizeof(int32_t));
  uint8_t* act = (uint8_t*)malloc(P);
  /* value of the previous interpolated frame per pixel (ORC_T_CROSSING) */
  int32_t* Iprev = (int32_t*)malloc(P * sizeof(int32_t));
  if (!Lprev || !Lcur || !R || !Fx || !Fy || !act || !Iprev) {
    free(Lprev); free(Lcur); free(R); free(Fx); free(Fy); free(act); free(Iprev);
    return -4;
  }
  const int crossing = c->event_time == ORC_T_CROSSING;

  /* Frame 0 sets the reference and emits nothing. */
  frame_to_log(c, lut, frames, Lprev);
  memcpy(R, Lprev, P * sizeof(int32_t));
  if (n_per_frame) n_per_frame[0] = 0;
  if (ev_per_frame) ev_per_frame[0] = 0;
  if (active_per_frame) active_per_frame[0] = 0;
  int64_t clamped = 0;

  int64_t n = 0;
  int64_t rc = 0;
  for (int32_t i = 1; i < n_frames; ++i) {
    int64_t t_prev = t_us[i - 1] - t_us[0];
    int64_t dt = t_us[i] - t_us[i - 1];
    if (dt <= 0) { rc = -2; break; }
    if (t_us[i] - t_us[0] > 4294967295LL) { rc = -3; break; }
    int64_t n_before = n;
    frame_to_log(c, lut, frames + (int64_t)i * fbytes, Lcur);

    /* Flow of frame i (i-1 -> i), read at the target pixel. */
    const float* fl = flows + (int64_t)i * P * 2;
    for (int64_t p = q_begin; p < q_end; ++p) {
      int32_t cl = 0;
      Fx[p] = orc_flow_q16(fl[2 * p], &cl);
      Fy[p] = orc_flow_q16(fl[2 * p + 1], &cl);
      if (p >= p_begin && p < p_end) clamped += cl;
    }

    /* Sec. III-B: pixels whose change from frame i-1 to frame i stays under
     * the activity threshold are disregarded (dense: every pixel counts). */
    int64_t n_active = 0;
    for (int64_t p = q_begin; p < q_end; ++p) {
      int32_t a = 1;
      if (c->mode == ORC_SPARSE) {
        int32_t cp = pixel_threshold(cpos_map, c->c_pos_q16, p);
        int32_t cn = pixel_threshold(cneg_map, c->c_neg_q16, p);
        int32_t cact = c->c_act_q16 >= 0 ? c->c_act_q16 : (cp < cn ? cp : cn);
        int64_t d = (int64_t)Lcur[p] - Lprev[p];
        if (d < 0) d = -d;
        a = d >= cact;
      }
      act[p] = (uint8_t)a;
      if (p >= p_begin && p < p_end) n_active += a;
    }

    int32_t N = c->substeps;
    if (N == 0) {
      int64_t m = 0;
      for (int64_t p = 0; p < P; ++p) {
        if (!act[p]) continue;
        int64_t f2 = (int64_t)Fx[p] * Fx[p] + (int64_t)Fy[p] * Fy[p];
        if (f2 > m) m = f2;
      }
      N = orc_adaptive_substeps(m, c->max_substeps);
    }

    /* RESET mode differences consecutive interpolated frames: the frame
     * before substep 1 is frame i-1 itself (Sec. III-A). */
    if (c->ref_mode == ORC_RESET) memcpy(R, Lprev, P * sizeof(int32_t));
    /* interpolated frame 0 of N is frame i-1 itself (zero offset, weight 0) */
    memcpy(Iprev, Lprev, P * sizeof(int32_t));

    for (int32_t k = 1; k <= N; ++k) {
      /* Q12 blend weight round-half-up(4096 k / N); w_N = 4096. */
      int64_t w = ((int64_t)k * 8192 + N) / (2 * (int64_t)N);
      uint32_t tk = (uint32_t)(t_prev + floordiv((int64_t)k * dt, N));
      int64_t tk1 = t_prev + floordiv((int64_t)(k - 1) * dt, N);  /* t_{k-1} */
      for (int32_t y = y0; y < y1; ++y) {
        for (int32_t x = 0; x < W; ++x) {
          int64_t p = (int64_t)y * W + x;
          if (!act[p]) continue;
          /* Interpolated frame k of N (Sec. III-A): the pixel's trajectory
           * passes x - (k/N) F in frame i-1 and x + (1 - k/N) F in frame i. */
          int64_t offx = floordiv((int64_t)Fx[p] * k, N);
          int64_t offy = floordiv((int64_t)Fy[p] * k, N);
          int64_t p0x = (int64_t)x * 65536 - offx, p0y = (int64_t)y * 65536 - offy;
          int64_t p1x = p0x + Fx[p], p1y = p0y + Fy[p];
          int64_t s0 = orc_bilinear(Lprev, W, H, p0x, p0y);
          int64_t s1 = orc_bilinear(Lcur, W, H, p1x, p1y);
          int64_t I = lerp_q12(s0, s1, w);

          int32_t cp = pixel_threshold(cpos_map, c->c_pos_q16, p);
          int32_t cn = pixel_threshold(cneg_map, c->c_neg_q16, p);
          int64_t D = I - R[p];
          /* the reference before this substep; the j-th level crossed is
           * Rb + j Cp (rising) or Rb - j Cn (falling) */
          int64_t Rb = R[p], ip = Iprev[p];
          Iprev[p] = (int32_t)I;
          if (c->ref_mode == ORC_RESET) {
            /* The two-case threshold equations of Sec. III-A, strict. */
            if (D > cp)
              emit(out, cap, &n, crossing ? (uint32_t)orc_crossing_time(tk1, tk, ip, I, Rb + cp, 1)
                                          : tk, x, y, 1);
            else if (D < -(int64_t)cn)
              emit(out, cap, &n, crossing ? (uint32_t)orc_crossing_time(tk1, tk, ip, I, Rb - cn, 0)
                                          : tk, x, y, 0);
            R[p] = (int32_t)I;
          } else {
            /* Reference-accumulating reading: every whole threshold crossed
             * by the difference is one event; the reference moves by it. */
            if (D >= cp) {
              int64_t m = D / cp;
              R[p] = (int32_t)(R[p] + m * cp);
              for (int64_t j = 1; j <= m; ++j)
                emit(out, cap, &n,
                     crossing ? (uint32_t)orc_crossing_time(tk1, tk, ip, I, Rb + j * cp, 1) : tk,
                     x, y, 1);
            } else if (-D >= cn) {
              int64_t m = (-D) / cn;
              R[p] = (int32_t)(R[p] - m * cn);
              for (int64_t j = 1; j <= m; ++j)
                emit(out, cap, &n,
                     crossing ? (uint32_t)orc_crossing_time(tk1, tk, ip, I, Rb - j * cn, 0) : tk,
                     x, y, 0);
            }
          }
        }
      }
    }
    if (n_per_frame) n_per_frame[i] = N;
    if (ev_per_frame) ev_per_frame[i] = n - n_before;
    if (active_per_frame) active_per_frame[i] = n_active;
    int32_t* tmp = Lprev; Lprev = Lcur; Lcur = tmp;
  }

  if (R_final) memcpy(R_final, R, P * sizeof(int32_t));
  if (clamped_total) *clamped_total = clamped;
  free(Lprev); free(Lcur); free(R); free(Fx); free(Fy); free(act); free(Iprev);
  return rc < 0 ? rc : n;
}

/*
 * Difference-frame interpolation (Sec. III-C).  From three consecutive
 * frames i-2, i-1, i the method forms two difference frames,
 *   D_{i-1} = L_{i-1} - L_{i-2},   D_i = L_i - L_{i-1}
 * (L the intensity table applied to the frame; Sec. III's linear difference
 * in ORC_LINEAR), takes the flow between the two difference frames (an
 * input, stored at index i), interpolates N difference frames between them
 * with the sampling and blend of the dense method (Sec. III-A), and
 * thresholds each interpolated difference frame with the two-case equations
 * of Sec. III-A (strict): the difference frames stand for the events, so
 * there is no reference state.  Events of substep k carry t_k between
 * t_{i-1} and t_i.  Frames 0 and 1 emit nothing (three frames are needed).
 * N: fixed, or adaptive from the largest flow of the frame (every pixel).
 */
int64_t orc_run_diff(const orc_config* c, int32_t n_frames, const uint8_t* frames,
                     const float* flows, const int64_t* t_us,
                     const uint16_t* cpos_map, const uint16_t* cneg_map,
                     orc_event* out, int64_t cap, int32_t* n_per_frame,
                     int64_t* ev_per_frame, int64_t* clamped_total) {
  if (!c || n_frames < 1 || !frames || !t_us || c->width < 1 || c->height < 1) return -1;
  if (c->channels != 1 && c->channels != 3) return -1;
  if (c->substeps < 0 || (c->substeps == 0 && c->max_substeps < 1)) return -1;
  if (n_frames > 2 && !flows) return -1;
  const int32_t W = c->width, H = c->height;
  const int64_t P = (int64_t)W * H;
  const int64_t fbytes = P * c->channels;

  int32_t lut[256];
  orc_lut(c->intensity, lut);

  int32_t* L2 = (int32_t*)malloc(P * sizeof(int32_t));   /* frame i-2 */
  int32_t* L1 = (int32_t*)malloc(P * sizeof(int32_t));   /* frame i-1 */
  int32_t* L0 = (int32_t*)malloc(P * sizeof(int32_t));   /* frame i */
  int32_t* Dp = (int32_t*)malloc(P * sizeof(int32_t));   /* D_{i-1} */
  int32_t* Dc = (int32_t*)malloc(P * sizeof(int32_t));   /* D_i */
  int32_t* Fx = (int32_t*)malloc(P * sizeof(int32_t));
  int32_t* Fy = (int32_t*)malloc(P * sizeof(int32_t));
  if (!L2 || !L1 || !L0 || !Dp || !Dc || !Fx || !Fy) {
    free(L2); free(L1); free(L0); free(Dp); free(Dc); free(Fx); free(Fy);
    return -4;
  }
  int64_t clamped = 0, n = 0, rc = 0;
  for (int32_t i = 0; i < n_frames; ++i) {
    if (i > 0) {
      if (t_us[i] <= t_us[i - 1]) { rc = -2; break; }
      if (t_us[i] - t_us[0] > 4294967295LL) { rc = -3; break; }
    }
    /* roll the three frames: L2 <- L1 <- L0 <- frame i */
    int32_t* tmp = L2; L2 = L1; L1 = L0; L0 = tmp;
    frame_to_log(c, lut, frames + (int64_t)i * fbytes, L0);
    if (n_per_frame) n_per_frame[i] = 0;
    if (ev_per_frame) ev_per_frame[i] = 0;
    if (i < 2) continue;
    int64_t n_before = n;
    for (int64_t p = 0; p < P; ++p) {
      Dp[p] = L1[p] - L2[p];
      Dc[p] = L0[p] - L1[p];
    }
    const float* fl = flows + (int64_t)i * P * 2;
    int64_t m = 0;
    for (int64_t p = 0; p < P; ++p) {
      int32_t cl = 0;
      Fx[p] = orc_flow_q16(fl[2 * p], &cl);
      Fy[p] = orc_flow_q16(fl[2 * p + 1], &cl);
      clamped += cl;
      int64_t f2 = (int64_t)Fx[p] * Fx[p] + (int64_t)Fy[p] * Fy[p];
      if (f2 > m) m = f2;
    }
    int32_t N = c->substeps > 0 ? c->substeps : orc_adaptive_substeps(m, c->max_substeps);
    int64_t t_prev = t_us[i - 1] - t_us[0];
    int64_t dt = t_us[i] - t_us[i - 1];
    for (int32_t k = 1; k <= N; ++k) {
      int64_t w = ((int64_t)k * 8192 + N) / (2 * (int64_t)N);
      uint32_t tk = (uint32_t)(t_prev + floordiv((int64_t)k * dt, N));
      for (int32_t y = 0; y < H; ++y) {
        for (int32_t x = 0; x < W; ++x) {
          int64_t p = (int64_t)y * W + x;
          /* interpolated difference frame k of N between D_{i-1} and D_i */
          int64_t offx = floordiv((int64_t)Fx[p] * k, N);
          int64_t offy = floordiv((int64_t)Fy[p] * k, N);
          int64_t p0x = (int64_t)x * 65536 - offx, p0y = (int64_t)y * 65536 - offy;
          int64_t p1x = p0x + Fx[p], p1y = p0y + Fy[p];
          int64_t s0 = orc_bilinear(Dp, W, H, p0x, p0y);
          int64_t s1 = orc_bilinear(Dc, W, H, p1x, p1y);
          int64_t I = lerp_q12(s0, s1, w);
          int32_t cp = pixel_threshold(cpos_map, c->c_pos_q16, p);
          int32_t cn = pixel_threshold(cneg_map, c->c_neg_q16, p);
          if (I > cp) emit(out, cap, &n, tk, x, y, 1);
          else if (I < -(int64_t)cn) emit(out, cap, &n, tk, x, y, 0);
        }
      }
    }
    if (n_per_frame) n_per_frame[i] = N;
    if (ev_per_frame) ev_per_frame[i] = n - n_before;
  }
  if (clamped_total) *clamped_total = clamped;
  free(L2); free(L1); free(L0); free(Dp); free(Dc); free(Fx); free(Fy);
  return rc < 0 ? rc : n;
}

/*
 * Accumulated event frame, the second output form of the methods (Fig. 1
 * caption: "a frame with the accumulated events"): every event with
 * t_begin <= t < t_end adds its polarity (+1 / -1) to its pixel.
 */
void orc_accumulate(const orc_event* ev, int64_t n, int32_t W, int32_t H, int64_t t_begin,
                    int64_t t_end, int32_t* frame) {
  for (int64_t i = 0; i < n; ++i) {
    int64_t t = ev[i].t;
    if (t < t_begin || t >= t_end) continue;
    int32_t x = ev[i].x, y = ev[i].yp >> 1;
    if (x >= W || y >= H) continue;
    frame[(int64_t)y * W + x] += (ev[i].yp & 1) ? 1 : -1;
  }
}
