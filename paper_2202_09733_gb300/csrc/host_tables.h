/* Host-side operator tables and mesh preprocessing of the frpmg library (C, binary128
 * tables rounded once to double; geometric factors evaluated in double with the fixed
 * fma-chain order that the device kernels also follow). */
#ifndef FRH_TABLES_H
#define FRH_TABLES_H
#ifdef __cplusplus
extern "C" {
#endif

#define FRH_MAXN 6

typedef struct {
    int p, n, g;
    double x[FRH_MAXN], w[FRH_MAXN];
    double D[FRH_MAXN][FRH_MAXN];
    double lm[FRH_MAXN], lp[FRH_MAXN], dlm[FRH_MAXN], dlp[FRH_MAXN];
    double gLd[FRH_MAXN], gRd[FRH_MAXN];
    double gLf, gRf;
    double gb[FRH_MAXN + 2][3], gdb[FRH_MAXN + 2][3];
} frh_tab;

void frh_make_tables(int p, int g, frh_tab *T);
void frh_make_transfer(int p0, int p1, double Gam[FRH_MAXN][FRH_MAXN], double Pi[FRH_MAXN][FRH_MAXN]);
/* M[a][i] = w_i phi_a(x_i): nodal values -> orthonormal Legendre coefficients (degree p) */
void frh_modal(int p, double M[FRH_MAXN][FRH_MAXN]);

/* geometric factors of one level: S, G [d][d][np][E]; invJ, Jdet [np][E];
 * Sf, Gf [d][d][nfp][E]  (arrays allocated by the caller) */
void frh_geometry(int d, int E, int qg, const double *gnodes, const frh_tab *T,
                  double *S, double *G, double *invJ, double *Jdet, double *Sf, double *Gf);

/* face-point pairs of one level, sorted by (kL, eL): pairs[P] = (eL, kL, eR, kR), bc[P];
 * returns the number of pairs (nfaces * n^(d-1)); -1 on an invalid face list */
int frh_pairs(int d, int n, int E, int nfaces, const int *faces, int *pairs, int *bc);

/* greedy distance-1 colouring of the element face graph; color[E]; returns #colours */
int frh_color(int E, int nfaces, const int *faces, int *color);
/* face-neighbour table nbr[f * E + e] (nf = 2d face slots): the element across face f of
 * e, or -1 for a boundary face, a face wrapping onto e itself and any face after the first
 * one reaching the same neighbour.  Returns 0, or -1 on a face naming a slot >= nf. */
int frh_neighbours(int E, int nf, int nfaces, const int *faces, int *nbr);
/* greedy distance-2 colouring from the neighbour table (no two elements within two face
 * steps share a colour); returns the number of colours, or -1 past 1024 colours */
int frh_color2(int E, int nf, const int *nbr, int *color);

#ifdef __cplusplus
}
#endif
#endif
