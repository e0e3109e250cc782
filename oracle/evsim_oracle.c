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

/*
 * Pyramidal Lucas-Kanade optical flow.  The paper computes the flow between
 * consecutive frames with OpenCV; its sparse and difference-frame
 * simulators use Lucas-Kanade (Sec. III-B: "any sparse optical flow
 * algorithm" on the selected pixels; Sec. IV-A, Figs. 3 and 4: "Sparse int.
 * w. LK", "Difference int. w. LK").  Lucas and Kanade (1981) take the flow
 * of a pixel as the least-squares solution of the linearised brightness
 * constancy equations Ix u + Iy v + It = 0 over a window around it,
 * iterated with the second frame resampled at the current estimate, and
 * coarse to fine over image pyramids for motions beyond the window.  The
 * paper fixes no parameters or precision; the reading here (O17):
 *   - images: 8-bit luma (BT.601 for RGB) times 16 (4 fractional bits);
 *     level l+1 is the 2 x 2 box average of level l, rounded half up, of
 *     size ((W_l + 1) / 2, (H_l + 1) / 2), reads clamped to the image;
 *   - gradients of the first frame: Ix = I(x+1, y) - I(x-1, y),
 *     Iy = I(x, y+1) - I(x, y-1) (twice the central difference), reads
 *     clamped; window: the (2r+1)^2 pixels p + (i, j), each coordinate
 *     clamped to the image;
 *   - G = sum of [Ix Ix, Ix Iy; Ix Iy, Iy Iy] over the window (int64);
 *     the pixel is tracked only if the smaller eigenvalue of G divided by
 *     the window area is at least min_eig, else its flow is its guess;
 *   - iteration: It(q) = J(q + g + v) - I(q), J sampled with the clamped
 *     bilinear of the simulator (Q16 position, 12-bit fractions, blends
 *     rounded half up); b = sum of (Ix It, Iy It) (int64); the update is
 *     -2 G^-1 b px (the factor 2: Ix is twice the derivative), evaluated
 *     in IEEE double in the order written below - the scale -2^17 / det G
 *     once per pixel and level, then each component's numerator times it -
 *     and rounded to Q16 (ties to even); v += update;
 *   - coarse to fine: the guess g of a pixel of level l is twice the flow
 *     of its parent (x / 2, y / 2) at level l + 1 (zero at the top);
 *     the flow of level 0 is the output, Q16 px, clamped to +-1024 px.
 */
static int32_t lk_at(const int32_t* P, int32_t W, int32_t H, int64_t x, int64_t y) {
  if (x < 0) x = 0;
  if (x > W - 1) x = W - 1;
  if (y < 0) y = 0;
  if (y > H - 1) y = H - 1;
  return P[y * W + x];
}

/* Clamp-to-edge bilinear sample of a Q4 level image at a Q16 position
 * (the same rounding as orc_bilinear). */
static int64_t lk_bilinear(const int32_t* P, int32_t W, int32_t H, int64_t px, int64_t py) {
  return orc_bilinear(P, W, H, px, py);
}

int orc_flow_lk(const orc_lk_config* c, int32_t W, int32_t H, int32_t channels,
                const uint8_t* f0, const uint8_t* f1, int32_t* flow) {
  if (!c || !f0 || !f1 || !flow || W < 1 || H < 1) return -1;
  if (channels != 1 && channels != 3) return -1;
  if (c->levels < 1 || c->levels > 8 || c->radius < 1 || c->radius > 7) return -1;
  if (c->iterations < 1 || c->iterations > 16) return -1;
  const int L = c->levels, r = c->radius;
  int32_t Ws[8], Hs[8];
  int32_t* I[8];
  int32_t* J[8];
  int64_t* D[8]; /* flow of each level, Q16, 2 per pixel */
  Ws[0] = W;
  Hs[0] = H;
  for (int l = 1; l < L; ++l) {
    Ws[l] = (Ws[l - 1] + 1) / 2;
    Hs[l] = (Hs[l - 1] + 1) / 2;
  }
  int fail = 0;
  for (int l = 0; l < L; ++l) {
    const int64_t n = (int64_t)Ws[l] * Hs[l];
    I[l] = (int32_t*)malloc(n * sizeof(int32_t));
    J[l] = (int32_t*)malloc(n * sizeof(int32_t));
    D[l] = (int64_t*)malloc(2 * n * sizeof(int64_t));
    if (!I[l] || !J[l] || !D[l]) fail = 1;
  }
  if (!fail) {
    /* level 0: luma times 16 */
    for (int64_t p = 0; p < (int64_t)W * H; ++p) {
      int32_t a, b;
      if (channels == 1) {
        a = f0[p];
        b = f1[p];
      } else {
        a = orc_luma(f0[3 * p], f0[3 * p + 1], f0[3 * p + 2]);
        b = orc_luma(f1[3 * p], f1[3 * p + 1], f1[3 * p + 2]);
      }
      I[0][p] = 16 * a;
      J[0][p] = 16 * b;
    }
    /* pyramids: 2 x 2 box averages, rounded half up */
    for (int l = 1; l < L; ++l) {
      for (int32_t y = 0; y < Hs[l]; ++y)
        for (int32_t x = 0; x < Ws[l]; ++x) {
          const int32_t* Pi = I[l - 1];
          const int32_t* Pj = J[l - 1];
          const int32_t w = Ws[l - 1], h = Hs[l - 1];
          int64_t si = (int64_t)lk_at(Pi, w, h, 2 * x, 2 * y) + lk_at(Pi, w, h, 2 * x + 1, 2 * y) +
                       lk_at(Pi, w, h, 2 * x, 2 * y + 1) + lk_at(Pi, w, h, 2 * x + 1, 2 * y + 1);
          int64_t sj = (int64_t)lk_at(Pj, w, h, 2 * x, 2 * y) + lk_at(Pj, w, h, 2 * x + 1, 2 * y) +
                       lk_at(Pj, w, h, 2 * x, 2 * y + 1) + lk_at(Pj, w, h, 2 * x + 1, 2 * y + 1);
          I[l][(int64_t)y * Ws[l] + x] = (int32_t)((si + 2) >> 2);
          J[l][(int64_t)y * Ws[l] + x] = (int32_t)((sj + 2) >> 2);
        }
    }
    const double area = (double)((2 * r + 1) * (2 * r + 1));
    const int64_t lim = (int64_t)1024 * 65536;
    /* coarse to fine */
    for (int l = L - 1; l >= 0; --l) {
      const int32_t w = Ws[l], h = Hs[l];
      const int32_t* Il = I[l];
      const int32_t* Jl = J[l];
      for (int32_t y = 0; y < h; ++y)
        for (int32_t x = 0; x < w; ++x) {
          int64_t gx = 0, gy = 0;
          if (l < L - 1) {
            const int64_t* Dp = D[l + 1];
            const int64_t pp = (int64_t)(y / 2) * Ws[l + 1] + (x / 2);
            gx = 2 * Dp[2 * pp];
            gy = 2 * Dp[2 * pp + 1];
          }
          /* structure tensor of the window */
          int64_t sxx = 0, sxy = 0, syy = 0;
          for (int j = -r; j <= r; ++j)
            for (int i = -r; i <= r; ++i) {
              int64_t qx = x + i, qy = y + j;
              if (qx < 0) qx = 0;
              if (qx > w - 1) qx = w - 1;
              if (qy < 0) qy = 0;
              if (qy > h - 1) qy = h - 1;
              const int64_t ix = (int64_t)lk_at(Il, w, h, qx + 1, qy) - lk_at(Il, w, h, qx - 1, qy);
              const int64_t iy = (int64_t)lk_at(Il, w, h, qx, qy + 1) - lk_at(Il, w, h, qx, qy - 1);
              sxx += ix * ix;
              sxy += ix * iy;
              syy += iy * iy;
            }
          const double a = (double)sxx, b = (double)sxy, d = (double)syy;
          const double det = a * d - b * b;
          const double tr = a + d, df = a - d;
          const double disc = sqrt(df * df + (4.0 * b) * b);
          const double lmin = (tr - disc) * 0.5;
          int64_t vx = 0, vy = 0;
          if (lmin / area >= c->min_eig && det > 0.0) {
            const double scale = -131072.0 / det;
            for (int k = 0; k < c->iterations; ++k) {
              int64_t bx = 0, by = 0;
              for (int j = -r; j <= r; ++j)
                for (int i = -r; i <= r; ++i) {
                  int64_t qx = x + i, qy = y + j;
                  if (qx < 0) qx = 0;
                  if (qx > w - 1) qx = w - 1;
                  if (qy < 0) qy = 0;
                  if (qy > h - 1) qy = h - 1;
                  const int64_t ix =
                      (int64_t)lk_at(Il, w, h, qx + 1, qy) - lk_at(Il, w, h, qx - 1, qy);
                  const int64_t iy =
                      (int64_t)lk_at(Il, w, h, qx, qy + 1) - lk_at(Il, w, h, qx, qy - 1);
                  const int64_t jv =
                      lk_bilinear(Jl, w, h, qx * 65536 + gx + vx, qy * 65536 + gy + vy);
                  const int64_t it = jv - lk_at(Il, w, h, qx, qy);
                  bx += ix * it;
                  by += iy * it;
                }
              const double ex = (double)bx, ey = (double)by;
              const double nx = d * ex - b * ey;
              const double ny = a * ey - b * ex;
              vx += (int64_t)nearbyint(nx * scale);
              vy += (int64_t)nearbyint(ny * scale);
              if (vx > lim) vx = lim;
              if (vx < -lim) vx = -lim;
              if (vy > lim) vy = lim;
              if (vy < -lim) vy = -lim;
            }
          }
          int64_t ox = gx + vx, oy = gy + vy;
          if (ox > lim) ox = lim;
          if (ox < -lim) ox = -lim;
          if (oy > lim) oy = lim;
          if (oy < -lim) oy = -lim;
          D[l][2 * ((int64_t)y * w + x)] = ox;
          D[l][2 * ((int64_t)y * w + x) + 1] = oy;
        }
    }
    for (int64_t p = 0; p < 2 * (int64_t)W * H; ++p) flow[p] = (int32_t)D[0][p];
  }
  for (int l = 0; l < L; ++l) {
    free(I[l]);
    free(J[l]);
    free(D[l]);
  }
  return fail ? -4 : 0;
}
