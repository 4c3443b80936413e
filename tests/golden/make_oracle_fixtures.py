"""Write tests/golden/oracle_regression.json: oracle outputs on small seeded
scenes, frozen so that any later change of the oracle's arithmetic shows up in
tests/test_golden.py. Calls only the oracle and the scene descriptors. Run from
the repository root: python tests/golden/make_oracle_fixtures.py"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import harm_scenes as hs  # noqa: E402
import oracle  # noqa: E402


def cases():
    yield "small_static_p0_p63", hs.small_static(), [0, 63]
    yield "wave_scene_6ch_p5", hs.ati_scene(n_pulses=16, nx=40, ny=24, n_range=1024), [5]
    yield "all_variants_p9", hs.uv_patterns(hs.choppy(hs.hetero_sea(
        hs.ar1_speckle(hs.ati_scene(n_pulses=24, nx=40, ny=24, n_range=1024), tau_s=0.03, doppler_hz=12.0),
        tile_m=32.0))), [9]


def main():
    out = {"note": "oracle IQ samples (re, im) at the 12 largest-magnitude bins of each listed pulse and channel"}
    for name, d, pulses in cases():
        iq = oracle.echo(d, pulses)
        entries = []
        for c in range(iq.shape[0]):
            for i, n in enumerate(pulses):
                row = iq[c, i]
                ks = np.argsort(-np.abs(row))[:12]
                for k in sorted(int(k) for k in ks):
                    entries.append([c, n, k, float(row[k].real), float(row[k].imag)])
        out[name] = entries
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_regression.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=0)
    print("wrote", path)


if __name__ == "__main__":
    main()
