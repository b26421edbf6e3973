/* oracle_internal.h -- shared declarations between the oracle's C files.
 * TEST INFRASTRUCTURE ONLY. */
#ifndef HPDR_ORACLE_INTERNAL_H
#define HPDR_ORACLE_INTERNAL_H
#include <stddef.h>
#include <stdint.h>

#define OMAXD 3
#define OMAXL 64

typedef struct {
    int d;
    size_t n[OMAXD];
    int L;
    size_t m[OMAXD][OMAXL + 1];      /* node count of dim k on level l */
    double *x[OMAXD][OMAXL + 1];     /* coordinate of each node (finest: i, or the given ones) */
} ohier;

/* coords: NULL (node i at coordinate i) or n[0] + ... + n[d-1] strictly
 * increasing finite coordinates, dimension 0 first */
int ohier_build(ohier *H, int d, const size_t *n, const double *coords);
void ohier_free(ohier *H);
size_t ohier_count(const ohier *H, int l);
size_t ocpos(size_t m, size_t mc, size_t j);
int ois_coarse(size_t m, size_t p);

#endif
