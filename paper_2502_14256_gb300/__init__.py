"""GB300-native structured-Gram kernel solves over randomized low-discrepancy points."""
