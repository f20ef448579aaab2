"""Writes seq_energy_layered_320x240x60.txt: the Eq. 1 energy (E_H, E_H~) of
the sequential-sweep oracle (Algorithm 1 as printed) after a whole
inpainting of the 320x240x60 layered workload, taken at level 0 after the
last search/reconstruction iteration and before the final best-patch step,
with the oracle's own evaluator. Calls only oracle/ and the seeded input
generator; about five minutes on one core.

    python tests/golden/make_seq_energy.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1503_05528_gb300 import synth  # noqa: E402

W, H, T, SPRITES, SPRITE_PX, HOLE, LEVELS, SEED = 320, 240, 60, 3, (20, 50), 0.08, 4, synth.BASE_SEED + 2
KEY_SEED = 1503


def main():
    clip = synth.layered_clip(W, H, T, SPRITES, SPRITE_PX, HOLE, LEVELS, SEED, name="layered_320x240x60")
    prm = O.Params(schedule="SEQ", seed=KEY_SEED)
    _, pyr, before_final = O.inpaint(clip.rgb, clip.mask, LEVELS, True, prm, return_levels=True)
    lv = pyr[0]
    e_h, e_ht = O.energy(before_final, lv.hole, lv.htilde, lv.phi)
    outer = [pyr[i].stats.get("outer") for i in range(LEVELS)]
    path = os.path.join(HERE, "seq_energy_layered_320x240x60.txt")
    with open(path, "w") as f:
        f.write("# Eq. 1 energy of the sequential-sweep oracle, layered_320x240x60 (seed %d, key %d),\n"
                % (SEED, KEY_SEED))
        f.write("# level 0 before the final step; written by tests/golden/make_seq_energy.py\n")
        f.write("E_H %.17g\nE_Htilde %.17g\n" % (e_h, e_ht))
        f.write("outer_per_level %s\n" % " ".join(str(o[0] if o else 0) for o in outer))
    print(open(path).read())


if __name__ == "__main__":
    main()
