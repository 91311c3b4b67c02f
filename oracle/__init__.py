"""FP64 CPU oracle of the SGML method: test infrastructure only (tests, smoke check, CPU baseline)."""
