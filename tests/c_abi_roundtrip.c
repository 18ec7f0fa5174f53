/* The library used from plain C through include/fetdpic.h only: a 4 x 4-cell
 * square mesh (two counter-clockwise triangles per cell, PEC walls), a uniform
 * B_z, two electrons, three FP64 Boris steps, then the particles read back.
 * Prints one line per particle: x y ux uy triangle, in %.17g.  Exit status 0
 * on success, 1 with the library's message on the first failing call.
 *
 * Build: cc -std=c99 -I include tests/c_abi_roundtrip.c -L <lib dir> -lfetdpic */
#include <stdio.h>
#include <string.h>

#include "fetdpic.h"

#define N 4

static int fail(fetdpic_ctx *ctx, const char *what, int rc)
{
    fprintf(stderr, "%s: status %d: %s\n", what, rc, ctx ? fetdpic_last_error(ctx) : "");
    if (ctx) fetdpic_destroy(ctx);
    return 1;
}

int main(void)
{
    double nodes[(N + 1) * (N + 1) * 2];
    int tri[N * N * 2 * 3];
    int k = 0;
    for (int j = 0; j <= N; ++j)
        for (int i = 0; i <= N; ++i) {
            nodes[2 * (j * (N + 1) + i)] = (double)i / N;
            nodes[2 * (j * (N + 1) + i) + 1] = (double)j / N;
        }
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
            const int a = j * (N + 1) + i, b = a + 1, c = a + N + 1, d = c + 1;
            tri[k++] = a; tri[k++] = b; tri[k++] = d;
            tri[k++] = a; tri[k++] = d; tri[k++] = c;
        }

    fetdpic_params p;
    memset(&p, 0, sizeof p);
    p.precision = FETDPIC_FP64;
    p.spai_level = 1;
    p.sort_interval = -1;

    fetdpic_instance in;
    memset(&in, 0, sizeof in);
    in.n_nodes = (N + 1) * (N + 1);
    in.nodes_xy = nodes;
    in.n_tri = N * N * 2;
    in.triangles = tri;
    in.dt = 1e-10;
    in.b0 = 0.05;

    fetdpic_ctx *ctx = NULL;
    int rc = fetdpic_create(&ctx, &p, 1, &in);
    if (rc) return fail(ctx, "fetdpic_create", rc);

    const double x[4] = {0.31, 0.42, 0.66, 0.71};
    const double u[4] = {2.0e7, -1.0e7, -3.0e7, 5.0e6};
    rc = fetdpic_load_particles(ctx, 0, -1.602176634e-19, 9.1093837015e-31, 2, x, u, NULL);
    if (rc) return fail(ctx, "fetdpic_load_particles", rc);
    rc = fetdpic_step(ctx, 3, FETDPIC_BORIS);
    if (rc) return fail(ctx, "fetdpic_step", rc);
    rc = fetdpic_sync(ctx);
    if (rc) return fail(ctx, "fetdpic_sync", rc);

    double xo[4], uo[4];
    int co[2];
    rc = fetdpic_read(ctx, 0, NULL, NULL, NULL, 0, xo, uo, co);
    if (rc) return fail(ctx, "fetdpic_read", rc);
    for (int q = 0; q < 2; ++q)
        printf("%.17g %.17g %.17g %.17g %d\n", xo[2 * q], xo[2 * q + 1], uo[2 * q], uo[2 * q + 1], co[q]);
    fetdpic_destroy(ctx);
    return 0;
}
