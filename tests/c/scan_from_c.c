/* A plain C99 program that scans through include/ac.h and libacgb300.so on
 * GPU 0, with no Python between it and the library: the worked example of
 * the paper's Fig. 1 (patterns AB, ABG, BEDE, EF on the input ABEDE: AB ends
 * at position 1, BEDE at position 4) through ac_scan, ac_scan_batch and the
 * serving calls, each checked record by record (built and run by
 * tests/test_abi_from_c.py). */
#include <stdio.h>
#include <string.h>
#include "ac.h"

static int check(const ac_result *r, const char *what) {
    static const uint32_t want[2][2] = {{1, 0}, {4, 2}};
    static const uint64_t want_counts[4] = {1, 0, 1, 0};
    if (r->num_matches != 2 || r->num_patterns != 4) {
        printf("%s: %llu matches\n", what, (unsigned long long)r->num_matches);
        return 1;
    }
    for (int i = 0; i < 2; ++i)
        if (r->matches[i].pos != want[i][0] || r->matches[i].pattern_id != want[i][1]) {
            printf("%s: match %d is (%u, %u)\n", what, i, r->matches[i].pos, r->matches[i].pattern_id);
            return 1;
        }
    for (int j = 0; r->counts && j < 4; ++j)
        if (r->counts[j] != want_counts[j]) {
            printf("%s: count %d is %llu\n", what, j, (unsigned long long)r->counts[j]);
            return 1;
        }
    return 0;
}

int main(void) {
    const char *p[4] = {"AB", "ABG", "BEDE", "EF"};
    const uint8_t *pats[4];
    uint32_t lens[4];
    for (int j = 0; j < 4; ++j) {
        pats[j] = (const uint8_t *)p[j];
        lens[j] = (uint32_t)strlen(p[j]);
    }
    ac_build_opts o;
    memset(&o, 0, sizeof(o));
    o.num_subsets = 1;
    o.device = 0;
    ac_automaton *a = NULL;
    if (ac_build(pats, lens, 4, &o, &a) != AC_OK) { printf("build: %s\n", ac_last_error()); return 1; }
    const uint8_t *text = (const uint8_t *)"ABEDE";
    ac_result r;
    if (ac_scan(a, text, 5, AC_U8, AC_HOST, NULL, &r) != AC_OK) { printf("scan: %s\n", ac_last_error()); return 2; }
    if (check(&r, "ac_scan")) return 3;
    ac_result_free(&r);

    const ac_automaton *as[1] = {a};
    ac_batch_item items[3];
    for (int i = 0; i < 3; ++i) {
        items[i].automaton = 0;
        items[i].fmt = AC_U8;
        items[i].text = text;
        items[i].n = 5;
    }
    ac_result outs[3];
    if (ac_scan_batch(as, 1, items, 3, AC_HOST, 0, NULL, outs) != AC_OK) { printf("batch: %s\n", ac_last_error()); return 4; }
    for (int i = 0; i < 3; ++i) {
        if (check(&outs[i], "ac_scan_batch")) return 5;
        ac_result_free(&outs[i]);
    }

    ac_server *srv = NULL;
    ac_serve_opts so;
    memset(&so, 0, sizeof(so));
    if (ac_serve_create(as, 1, &so, &srv) != AC_OK) { printf("serve: %s\n", ac_last_error()); return 6; }
    uint64_t t[4];
    for (int i = 0; i < 4; ++i)
        if (ac_serve_submit(srv, 0, text, 5, AC_U8, &t[i]) != AC_OK) return 7;
    for (int i = 0; i < 4; ++i) {
        if (ac_serve_wait(srv, t[i], 60000, &r) != AC_OK) { printf("wait: %s\n", ac_last_error()); return 8; }
        if (check(&r, "ac_serve_wait")) return 9;
        ac_result_free(&r);
    }
    ac_serve_destroy(srv);
    ac_free(a);
    printf("ok\n");
    return 0;
}
