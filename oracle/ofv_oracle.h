/*
 * FP64 CPU oracle of the dense optical-flow velocimetry estimator.
 * TEST INFRASTRUCTURE ONLY: called by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the estimator.  Shares nothing with
 * the CUDA path.  Definitions and citations are in ofv_oracle.c.
 */
#ifndef OFV_ORACLE_H
#define OFV_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int psl;              /* pyramid sub-levels; levels 0..psl (PSL = 0: no pyramid) */
    int kr;               /* kernel radius: window (2KR+1)^2 */
    int it;               /* Gauss-Newton iterations per level */
    int nr;               /* normalization radius; 0 = off */
    int bits;             /* > 0: inputs are counts, I = raw / (2^bits - 1) */
    int prefilter;        /* 1: 5x5 correlation with w25 after normalization */
    const double *w25;    /* row-major 5x5 weights (used when prefilter = 1) */
    double eps_rel;       /* relative determinant guard */
    double eps_abs;       /* absolute trace guard */
    double eps_n;         /* normalization floor */
    int increment_form;   /* 1: V = V0(m) + H^-1 sum G(-It) instead of the direct form */
    double win_sigma;     /* > 0: Gaussian window weights exp(-(a^2+b^2)/(2 sigma^2)); 0: uniform box */
    const double *u_init; /* initial level-0 field (warm start), or NULL for V = 0 at the coarsest level */
    const double *v_init;
    const unsigned char *mask; /* level-0 region mask (nonzero = valid), or NULL: masked pixels' products are
                                  left out of every window sum and their output is NaN */
} orc_params;

void orc_scale(int64_t n, const double *raw, int bits, double *out);
void orc_normalize(int H, int W, const double *I, int nr, double eps_n, double *out);
void orc_prefilter(int H, int W, const double *I, const double *w25, double *out);
void orc_reduce(int H, int W, const double *P, double *out);
double orc_bilinear(const double *P, int H, int W, double px, double py);
void orc_central_diff(int H, int W, const double *P, double *Dx, double *Dy);
void orc_box_sum(int H, int W, const double *in, int kr, double *out);
void orc_window_sum(int H, int W, const double *in, int kr, double sigma, double *out);
void orc_upsample(int Hc, int Wc, const double *uc, const double *vc, int H, int W,
                  double *u, double *v);
int orc_iterate(int H, int W, const double *P1, const double *P2, const double *u0,
                const double *v0, int kr, double win_sigma, double eps_rel, double eps_abs,
                int increment_form, const unsigned char *mask, double *u, double *v, double *ndet,
                unsigned char *guarded);
void orc_decimate_mask(int H, int W, const unsigned char *mask, int level, unsigned char *out);
void orc_decimate_field(int H, int W, const double *u, const double *v, int level, double *uc, double *vc);
void orc_level_sizes(int H, int W, int psl, int *Hs, int *Ws);
int orc_ingest(int H, int W, const double *raw, const orc_params *p, double *out);
int orc_pyramid(int H, int W, const double *raw, const orc_params *p, double *out);
int orc_flow(int H, int W, const double *raw1, const double *raw2, const orc_params *p,
             double *u, double *v, double *ndet, unsigned char *guard0);
void orc_vorticity(int H, int W, const double *u, const double *v, double *omega);
int64_t orc_recirculation_count(int H, int W, const double *u, const unsigned char *mask);
/* threads the OpenMP loops of the oracle run on (1 when built without OpenMP) */
int orc_num_threads(void);
/* reverse mode (ofv_oracle_adjoint.c): gw25 accumulates (zero it first) */
int orc_flow_grad(int H, int W, const double *raw1, const double *raw2, const orc_params *p,
                  const double *gu, const double *gv, double *g1, double *g2, double *gw25,
                  double *u, double *v);

#ifdef __cplusplus
}
#endif
#endif
